"""A small uneven batch solved once with lq_batch_cg_solve (even-odd, FP16 inner), run in a
process of its own so that the library reads LQCD_TUNE_CACHE (the autotuner's cache file) at
its first tuning; prints the worst true residual and the solve's wall time as JSON."""
import json
import os
import sys
import time

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2001_07557_gb300 import inputs, lqcd  # noqa: E402

SHAPES = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8)]


def main():
    hs, bs, xs = [], [], []
    for i, dims in enumerate(SHAPES):
        V = int(np.prod(dims))
        U = torch.from_numpy(inputs.gauge_field(dims, "smooth", seed=1500 + i)).cuda()
        hs.append(lqcd.lq_create(lqcd.make_params(dims, mass=0.05), U))
        bs.append(torch.from_numpy(inputs.gaussian_spinor(V // 2, seed=2500 + i, nrhs=2)).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=2, tol=1e-10,
                             inner=lqcd.LQ_F16)
    t0 = time.perf_counter()
    rc, st = lqcd.lq_batch_cg_solve(hs, xs, bs, cp)
    dt = time.perf_counter() - t0
    print(json.dumps({"rc": rc, "worst": max(s.true_rel_residual for s in st), "seconds": dt,
                      "x0": [float(x.abs().sum()) for x in xs]}))
    for h in hs:
        lqcd.lq_destroy(h)


if __name__ == "__main__":
    main()
