"""Write tests/golden/oracle_4444.json from the CPU oracle only.

The fixture is a drift check for the oracle: the 4^4 workload (random SU(3)
links, seed 1000; Gaussian source, seed 2000; m = 0.1, r = 1, antiperiodic in
time) is pushed through D, D^dag and CG on D^dag D to 1e-12, and a handful of
sampled output entries are stored with a hash of the inputs, so that a change
in the input generator is reported as such and not as an oracle change.

Run from the repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2001_07557_gb300 import inputs  # noqa: E402

DIMS = (4, 4, 4, 4)
MASS = 0.1
SAMPLES = [0, 1, 7, 100, 255]


def workload():
    U = inputs.gauge_field(DIMS, "random", seed=1000)
    eta = inputs.gaussian_spinor(256, seed=2000)
    return U, eta


def input_hash(U, eta):
    h = hashlib.sha256()
    h.update(np.round(U, 12).tobytes())
    h.update(np.round(eta, 12).tobytes())
    return h.hexdigest()


def pack(v):
    return [[float(z.real), float(z.imag)] for z in v]


def compute():
    U, eta = workload()
    prm = oracle.params(DIMS, mass=MASS)
    d = oracle.wilson_dslash(eta, U, DIMS, MASS)
    dd = oracle.wilson_dslash(eta, U, DIMS, MASS, dagger=True)
    b = dd
    x, it, res, rc = oracle.cg(oracle.OP_WILSON, b, U, prm, 1e-12)
    out = {
        "input_sha256": input_hash(U, eta),
        "dims": list(DIMS), "mass": MASS, "bc": [1, 1, 1, -1],
        "samples": SAMPLES,
        "D_eta": pack(d[SAMPLES].reshape(-1)),
        "Ddag_eta": pack(dd[SAMPLES].reshape(-1)),
        "norm_D_eta": float(np.linalg.norm(d)),
        "cg_iterations": int(it),
        "cg_x": pack(x[SAMPLES].reshape(-1)),
    }
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_4444.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=0)
    print("wrote", path)
