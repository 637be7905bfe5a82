"""GPU parity: the even-odd (4-d parity) preconditioned domain wall -- the
Schur complement Mhat = M5 - M_eo M5^{-1} M_oe, source preparation, odd-half
reconstruction and CG on Mhat^dag Mhat -- against the FP64 oracle.

Tolerances as for the domain-wall hop (three hop-sized steps): FP64 1e-12
norm-wise and element-wise of the largest element; FP32 3e-6 / 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, max_err, native_buffer, rel_err
from paper_2001_07557_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQ_F64: (1e-12, 1e-12), lqcd.LQ_F32: (3e-6, 2e-5)}
M5, MF = 1.8, 0.05


def check(got, want, prec):
    tn, te = TOL[prec]
    assert rel_err(got, want) <= tn, (rel_err(got, want), tn)
    assert max_err(got, want) <= te, (max_err(got, want), te)


def half5(dims, Ls, seed):
    return inputs.gaussian_spinor(int(np.prod(dims)) // 2, seed=seed, nrhs=Ls)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("dims,Ls", [((4, 4, 2, 4), 4), ((2, 6, 4, 2), 6), ((4, 2, 2, 4), 1)])
def test_schur_apply(prec, native, dims, Ls):
    U = inputs.gauge_field(dims, "random", seed=1101)
    x = half5(dims, Ls, 2101)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=MF) as H:
        for dag in (False, True):
            want = oracle.dwf_schur(x, U, dims, Ls, M5, MF, dagger=dag)
            xd = dev(x, prec)
            y = torch.empty_like(xd)
            if native:
                nat = lqcd.LQ_NATIVE | prec
                xn = native_buffer(H.h, prec, lqcd.LQ_EVEN, Ls)
                yn = native_buffer(H.h, prec, lqcd.LQ_EVEN, Ls)
                lqcd.lq_convert(H.h, xn, nat, xd, prec, lqcd.LQ_EVEN, Ls)
                lqcd.dwf_schur_apply(H.h, yn, xn, nat, dag)
                lqcd.lq_convert(H.h, y, prec, yn, nat, lqcd.LQ_EVEN, Ls)
            else:
                lqcd.dwf_schur_apply(H.h, y, xd, prec, dag)
            check(host(y), want, prec)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
def test_prepare_and_reconstruct(prec):
    dims, Ls = (4, 4, 2, 4), 5
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1102)
    eta = inputs.gaussian_spinor(V, seed=2102, nrhs=Ls)
    xe = half5(dims, Ls, 2103)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=MF) as H:
        ed = dev(eta, prec)
        bh = torch.empty((Ls, V // 2, 4, 3), dtype=ed.dtype, device="cuda")
        lqcd.dwf_eo_prepare(H.h, bh, ed, prec)
        check(host(bh), oracle.dwf_eo_prepare(eta, U, dims, Ls, M5, MF), prec)
        psi = torch.empty_like(ed)
        lqcd.dwf_eo_reconstruct(H.h, psi, dev(xe, prec), ed, prec)
        check(host(psi), oracle.dwf_eo_reconstruct(xe, eta, U, dims, Ls, M5, MF), prec)


@pytest.mark.parametrize("mode", ["fp64", "mixed_f32"])
def test_eo_cg_solves_the_full_domain_wall_system(mode):
    """D_dw psi = eta through the Schur complement: prepare the source, CG on
    Mhat^dag Mhat x_e = Mhat^dag bhat_e to 1e-10, reconstruct psi; psi must
    solve the full system (checked with the oracle's D_dw)."""
    dims, Ls = (4, 4, 4, 4), 6
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1103)
    eta = inputs.gaussian_spinor(V, seed=2104, nrhs=Ls)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=MF) as H:
        ed = dev(eta)
        bh = torch.empty((Ls, V // 2, 4, 3), dtype=ed.dtype, device="cuda")
        lqcd.dwf_eo_prepare(H.h, bh, ed, lqcd.LQ_F64)
        b = torch.empty_like(bh)
        lqcd.dwf_schur_apply(H.h, b, bh, lqcd.LQ_F64, True)
        x = torch.zeros_like(b)
        m = lqcd.LQ_CG_PLAIN if mode == "fp64" else lqcd.LQ_CG_MIXED
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_EO_NORMAL, m, lqcd.LQ_F64, tol=1e-10, inner=lqcd.LQ_F32)
        rc, st = lqcd.cg_solve(H.h, x, b, cp)
        assert rc == 0 and st[0].true_rel_residual < 1e-10
        psi = torch.empty_like(ed)
        lqcd.dwf_eo_reconstruct(H.h, psi, x, ed, lqcd.LQ_F64)
        p = host(psi)
    # the normal-equation residual 1e-10 bounds |D psi - eta|/|eta| by about cond(Mhat) * 1e-10
    assert rel_err(oracle.dwf_dslash(p, U, dims, Ls, M5, MF), eta) < 1e-7
    xo, _, _, _ = oracle.cg(oracle.OP_DWF_EO, host(b), U, oracle.params(dims, Ls=Ls, M5=M5, mf=MF), 1e-12)
    assert rel_err(host(x), xo) < 1e-7


def test_eo_rejects_half_precision_and_block():
    dims, Ls = (4, 4, 2, 4), 2
    U = inputs.gauge_field(dims, "unit")
    with Handle(dims, U, Ls=Ls, M5=M5, mf=MF) as H:
        n = lqcd.lq_field_bytes(H.h, lqcd.LQ_NATIVE | lqcd.LQ_F16, lqcd.LQ_EVEN, Ls)
        a, b = (torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(2))
        with pytest.raises(lqcd.LqError):
            lqcd.dwf_schur_apply(H.h, b, a, lqcd.LQ_NATIVE | lqcd.LQ_F16)
        x = torch.zeros((Ls, 64, 4, 3), dtype=torch.complex128, device="cuda")
        for m, inner in ((lqcd.LQ_CG_MIXED, lqcd.LQ_F16), (lqcd.LQ_CG_BLOCK, lqcd.LQ_F32)):
            cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_EO_NORMAL, m, lqcd.LQ_F64, tol=1e-10, inner=inner)
            rc, _ = lqcd.cg_solve(H.h, x, torch.ones_like(x), cp, check=False)
            assert rc == -1  # LQ_ERR_ARG


@pytest.mark.slow
def test_full_size_schur_f32():
    """16^4 x Ls 16 (the benchmark's domain-wall workload), FP32 native, both daggers."""
    dims, Ls = (16, 16, 16, 16), 16
    U = inputs.gauge_field(dims, "smooth", seed=1004)
    x = half5(dims, Ls, 2004)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=0.01) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        xn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_EVEN, Ls)
        yn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_EVEN, Ls)
        xd = dev(x, lqcd.LQ_F32)
        lqcd.lq_convert(H.h, xn, nat, xd, lqcd.LQ_F32, lqcd.LQ_EVEN, Ls)
        y = torch.empty_like(xd)
        for dag in (False, True):
            lqcd.dwf_schur_apply(H.h, yn, xn, nat, dag)
            lqcd.lq_convert(H.h, y, lqcd.LQ_F32, yn, nat, lqcd.LQ_EVEN, Ls)
            check(host(y), oracle.dwf_schur(x, U, dims, Ls, M5, 0.01, dagger=dag), lqcd.LQ_F32)
