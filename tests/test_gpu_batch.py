"""lq_batch_cg_solve: independent lattices of different sizes in one
persistent, graph-captured solve, against the per-lattice solver and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, rel_err
from paper_2001_07557_gb300 import inputs
from paper_2001_07557_gb300 import lqcd

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 6, 6, 6), (4, 4, 8, 8), (8, 8, 8, 8)]


@pytest.mark.parametrize("inner", [lqcd.LQ_F16, lqcd.LQ_BF16, lqcd.LQ_F32])
@pytest.mark.parametrize("op", [lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_OP_WILSON_NORMAL])
def test_uneven_batch_mixed(inner, op):
    nr = 3
    m = 0.05
    Hs, bs, xs, want = [], [], [], []
    try:
        for i, dims in enumerate(SHAPES):
            V = int(np.prod(dims))
            U = inputs.gauge_field(dims, "smooth", seed=1100 + i)
            n = V // 2 if op == lqcd.LQ_OP_WILSON_EO_NORMAL else V
            b = inputs.gaussian_spinor(n, seed=2100 + i, nrhs=nr)
            H = Handle(dims, U, mass=m)
            Hs.append(H)
            bs.append(dev(b))
            xs.append(torch.zeros_like(bs[-1]))
            prm = oracle.params(dims, mass=m)
            oop = oracle.OP_WILSON_EO if op == lqcd.LQ_OP_WILSON_EO_NORMAL else oracle.OP_WILSON
            want.append([oracle.cg(oop, b[k], U, prm, 1e-12)[0] for k in range(nr)])
        cp = lqcd.make_cg_params(op, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=nr, tol=1e-10, inner=inner)
        rc, st = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, cp)
        assert rc == 0
        for i in range(len(SHAPES)):
            xg = host(xs[i])
            for k in range(nr):
                assert st[i * nr + k].true_rel_residual < 1e-10
                assert rel_err(xg[k], want[i][k]) < 1e-7
        # a second solve reuses the tuned launch shape and gives the same answer
        xs2 = [torch.zeros_like(b) for b in bs]
        rc, st2 = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs2, bs, cp)
        assert rc == 0
        for i in range(len(SHAPES)):
            assert torch.allclose(xs2[i], xs[i], rtol=0, atol=1e-9 * float(xs[i].abs().max()))
    finally:
        for H in Hs:
            H.close()


def test_batch_plain_fp32_and_argument_checks():
    dims_list = [(4, 4, 4, 4), (4, 4, 4, 8)]
    Hs, bs, xs = [], [], []
    try:
        for i, dims in enumerate(dims_list):
            V = int(np.prod(dims))
            H = Handle(dims, inputs.gauge_field(dims, "smooth", seed=1200 + i), mass=0.1)
            Hs.append(H)
            bs.append(dev(inputs.gaussian_spinor(V // 2, seed=2200 + i, nrhs=2), lqcd.LQ_F32))
            xs.append(torch.zeros_like(bs[-1]))
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F32, nrhs=2, tol=1e-5)
        rc, st = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, cp)
        assert rc == 0 and all(s.status == 0 for s in st)
        # FP64 plain is not a batched mode; DWF is not batched; the same handle twice is refused
        for bad in (lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, nrhs=2),
                    lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=2)):
            rc, _ = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, bad, check=False)
            assert rc == -1
        rc, _ = lqcd.lq_batch_cg_solve([Hs[0].h, Hs[0].h], xs, bs, cp, check=False)
        assert rc == -1
    finally:
        for H in Hs:
            H.close()


def test_uneven_batch_with_a_zero_right_hand_side():
    """One right-hand side of one lattice is zero: it is finished from the start
    (solution zero, no iterations), and the FP32 middle level of the others is
    unaffected."""
    nr, m = 2, 0.05
    Hs, bs, xs = [], [], []
    try:
        for i, dims in enumerate(SHAPES[:3]):
            V = int(np.prod(dims))
            U = inputs.gauge_field(dims, "smooth", seed=1150 + i)
            b = inputs.gaussian_spinor(V // 2, seed=2150 + i, nrhs=nr)
            if i == 1:
                b[0] = 0
            Hs.append(Handle(dims, U, mass=m))
            bs.append(dev(b))
            xs.append(torch.full_like(bs[-1], 3.0))
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=nr, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, cp)
        assert rc == 0
        assert np.all(host(xs[1])[0] == 0) and st[1 * nr + 0].iters == 0
        for g, s_ in enumerate(st):
            if g != nr:
                assert s_.true_rel_residual < 1e-10
    finally:
        for H in Hs:
            H.close()


def test_autotuner_cache_file_holds_a_tile_size_per_lattice(tmp_path):
    """The batch autotuner writes one line per batch shape to LQCD_TUNE_CACHE: a key naming the
    device model and the lattices, the resident blocks, the lattice count and each lattice's
    tiles per work item (1, 2, 4 or 8).  A second process reads the line back instead of tuning
    and solves to the same result."""
    import json
    import os
    import subprocess
    import sys

    cache = tmp_path / "tune.txt"
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache))
    script = os.path.join(os.path.dirname(__file__), "batch_tune_workload.py")
    runs = []
    for _ in range(2):
        out = subprocess.run([sys.executable, script], env=env, capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr
        runs.append(json.loads(out.stdout.strip().splitlines()[-1]))
    assert all(r["rc"] == 0 and r["worst"] < 1e-10 for r in runs)
    assert runs[0]["x0"] == runs[1]["x0"]  # same shape, same arithmetic: the same solution
    lines = cache.read_text().split("\n")
    lines = [ln for ln in lines if ln.strip()]
    assert len(lines) == 1
    tok = lines[0].split()
    key, blocks, nlat, mult = tok[0], int(tok[1]), int(tok[2]), [int(v) for v in tok[3:]]
    name = torch.cuda.get_device_name(0).replace(" ", "_").replace(":", "_")
    assert key.startswith("batch:" + name[:63] + ":sm") and key.endswith(":4x4x4x4:6x6x6x6:8x8x8x8")
    assert blocks >= 1 and nlat == 3 and len(mult) == 3 and all(m in (1, 2, 4, 8) for m in mult)
