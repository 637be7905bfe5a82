"""The index-checked build: liblqcd_checked.so, compiled with -DLQ_INDEX_CHECK,
compares every neighbour index the hop kernels compute with its parity block
before use (see lq_index_faults).  Run on the shapes of
tests/index_check_workload.py in a process of its own, the kernels must report
no index out of range and still give the oracle's results.  A CPU test checks
that the normal build reports itself as unchecked."""
import json
import os
import subprocess
import sys

import pytest

from paper_2001_07557_gb300 import build, lqcd

WORKLOAD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "index_check_workload.py")

# largest relative error allowed per kind of launch: the per-precision tolerances
# of the parity tests (FP64 1e-12, FP32 2e-6, FP16 2e-3, BF16 1.5e-2), the solvers' 1e-9
TOL = {"p0": 1e-12, "p1": 2e-6, "p2": 2e-3, "p3": 1.5e-2, "kind": 2e-3, "mobius": 1e-12, "slices": 2e-6,
       "cg": 1e-9, "batch": 1e-9}


def tolerance(kind):
    for key, tol in TOL.items():
        if key in kind:
            return tol
    raise KeyError(kind)


@pytest.mark.gpu
def test_checked_build_reports_no_index_out_of_range():
    lib = build.build(checked=True)
    env = dict(os.environ, LQCD_LIBRARY=lib)
    r = subprocess.run([sys.executable, WORKLOAD], env=env, capture_output=True, text=True, timeout=1200,
                       cwd=os.path.dirname(os.path.dirname(WORKLOAD)))
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["checked"] == 1
    assert res["faults"] == 0, res
    assert res["launches"] > 50
    for kind, err in res["errors"].items():
        assert err < tolerance(kind), (kind, err)


def test_normal_build_is_unchecked():
    if not os.path.exists(lqcd.LIB_PATH):
        build.build()
    count, first, checked = lqcd.lq_index_faults()
    assert (count, first, checked) == (0, -1, 0)
