"""The oracle reproduces its stored 4^4 fixture (tests/golden/oracle_4444.json)."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def load_maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_matches_golden(orc):
    mk = load_maker()
    stored = json.load(open(os.path.join(HERE, "golden", "oracle_4444.json")))
    U, eta = mk.workload()
    if mk.input_hash(U, eta) != stored["input_sha256"]:
        pytest.skip("input generator stream differs from the one the fixture was written with")
    now = mk.compute()
    for key in ("D_eta", "Ddag_eta", "cg_x"):
        a = np.array(now[key])
        b = np.array(stored[key])
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), key
    assert abs(now["norm_D_eta"] - stored["norm_D_eta"]) <= 1e-12 * stored["norm_D_eta"]
    assert abs(now["cg_iterations"] - stored["cg_iterations"]) <= 1
