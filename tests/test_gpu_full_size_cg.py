"""Full-size solver parity at the benchmark's configurations, through the
properties that hold at any size: the FP64 oracle's own normal operator
applied to each returned solution must reproduce the right-hand side to the
solver tolerance (the oracle's CG itself would take minutes at this size).

  32^4, m = 0.01, smooth links: the mixed solve (FP64 outer, FP32 middle,
  FP16 inner) and the plain FP64 solve of Mhat^dag Mhat x = b to 1e-10: the
  oracle's |b - A x| / |b| is at most 1e-10 for both, and they agree (both
  within cond * 1e-10 of the exact solution).
  16^3 x 32, m = 0.05: the FP64 even-odd solve and the mixed one with FP32
  inner solves.
  16^4 x Ls 16: the domain-wall solve refined in FP64, unpreconditioned and
  even-odd, mapped back to eta by the oracle's D_dw.
  24^3 x 48: the 12-source batched mixed solve, three solutions mapped back to
  their sources by the oracle's D.
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
        # |b - A x| / |b| from the oracle's own operator: the stated target, 1e-10
        assert rel_err(oracle.apply_normal(oracle.OP_WILSON_EO, x, U, prm), b) <= 1e-10
    assert rel_err(x_mixed, x_fp64) < 1e-7


def test_domain_wall_refined_solves_at_full_size():
    """16^4 x Ls 16, M5 = 1.8, mf = 0.01: D_dw psi = eta through CG on D_dw^dag D_dw
    (FP64 outer, FP32 inner) and through the even-odd Schur complement; the
    oracle's D_dw maps both solutions back to eta."""
    dims, Ls, M5, mf = (16, 16, 16, 16), 16, 1.8, 0.01
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1004)
    eta = inputs.gaussian_spinor(V, seed=2004, nrhs=Ls)
    b = oracle.dwf_dslash(eta, U, dims, Ls, M5, mf, dagger=True)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=mf) as H:
        bd = dev(b)
        x = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                                 inner=lqcd.LQ_F32, inner_tol=1e-6)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp)
        assert rc == 0 and st[0].true_rel_residual < 1e-10
        psi_full = host(x)
        ed = dev(eta)
        bh = torch.empty((Ls, V // 2, 4, 3), dtype=ed.dtype, device="cuda")
        lqcd.dwf_eo_prepare(H.h, bh, ed, lqcd.LQ_F64)
        be = torch.empty_like(bh)
        lqcd.dwf_schur_apply(H.h, be, bh, lqcd.LQ_F64, True)
        xe = torch.zeros_like(be)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                                 inner=lqcd.LQ_F32, inner_tol=1e-6)
        rc, st = lqcd.cg_solve(H.h, xe, be, cp)
        assert rc == 0 and st[0].true_rel_residual < 1e-10
        psi = torch.empty_like(ed)
        lqcd.dwf_eo_reconstruct(H.h, psi, xe, ed, lqcd.LQ_F64)
        psi_eo = host(psi)
    for p in (psi_full, psi_eo):
        assert rel_err(oracle.dwf_dslash(p, U, dims, Ls, M5, mf), eta) < 1e-8


def test_twelve_point_sources_batched_mixed_at_full_size():
    """24^3 x 48, m = 0.02, 12 point sources: the batched mixed solve (FP16 inner) of
    D^dag D x = D^dag b; the oracle's D maps every solution back to its source."""
    dims, m = (24, 24, 24, 48), 0.02
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1003)
    src = inputs.point_sources(V)
    with Handle(dims, U, mass=m) as H:
        sd = dev(src)
        bd = torch.empty_like(sd)
        lqcd.dslash_dag_apply(H.h, bd, sd, lqcd.LQ_F64, lqcd.LQ_FULL, nrhs=12)
        x = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=12, tol=1e-10,
                                 maxiter=40000, inner=lqcd.LQ_F16)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp)
        assert rc == 0 and max(s.true_rel_residual for s in st) < 1e-10
        xs = host(x)
    for k in (0, 5, 11):
        assert rel_err(oracle.wilson_dslash(xs[k], U, dims, m), src[k]) < 1e-8
