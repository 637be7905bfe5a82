"""Full-size solver parity at the benchmark's configurations, through the
properties that hold at any size: the FP64 oracle's own normal operator
applied to each returned solution must reproduce the right-hand side to the
solver tolerance (the oracle's CG itself would take minutes at this size).

  32^4, m = 0.01, smooth links: the mixed solve (FP64 outer, FP32 middle,
  FP16 inner) and the plain FP64 solve of Mhat^dag Mhat x = b to 1e-10, and
  their difference (both within cond * 1e-10 of the exact solution).
  16^3 x 32, m = 0.05: the FP64 even-odd solve and the mixed one with FP32
  inner solves.
"""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, rel_err
from paper_2001_07557_gb300 import inputs, lqcd

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def solve(H, b, mode, inner):
    bd = dev(b)
    x = torch.zeros_like(bd)
    cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, mode, lqcd.LQ_F64, tol=1e-10, maxiter=40000, inner=inner)
    rc, st = lqcd.cg_solve(H.h, x, bd, cp)
    assert rc == 0, lqcd.STATUS[rc]
    assert st[0].true_rel_residual < 1e-10
    return host(x)


@pytest.mark.parametrize("dims,mass,seed,inner", [((32, 32, 32, 32), 0.01, 1002, lqcd.LQ_F16),
                                                  ((16, 16, 16, 32), 0.05, 1001, lqcd.LQ_F32)])
def test_even_odd_solves_at_full_size(dims, mass, seed, inner):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=seed)
    b = inputs.gaussian_spinor(V // 2, seed=2002)
    with Handle(dims, U, mass=mass) as H:
        x_mixed = solve(H, b, lqcd.LQ_CG_MIXED, inner)
        x_fp64 = solve(H, b, lqcd.LQ_CG_PLAIN, lqcd.LQ_F32)
    prm = oracle.params(dims, mass=mass)
    for x in (x_mixed, x_fp64):
        # |b - A x| / |b| from the oracle's operator; 2e-10 leaves room for the rounding of one
        # FP64 Mhat^dag Mhat application on each side
        assert rel_err(oracle.apply_normal(oracle.OP_WILSON_EO, x, U, prm), b) < 2e-10
    assert rel_err(x_mixed, x_fp64) < 1e-7
