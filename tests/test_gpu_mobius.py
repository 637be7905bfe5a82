"""GPU parity: the Moebius domain-wall operator D_M = (b5 D_W + 1) + (c5 D_W - 1) S,
its even-odd Schur complement Mhat = M5_M - M_eo M5_M^{-1} M_oe (source
preparation, odd-half reconstruction) and CG on D_M^dag D_M and Mhat^dag Mhat,
against the FP64 oracle.  Tolerances as for the domain-wall hop: FP64 1e-12,
FP32 3e-6 norm-wise / 2e-5 element-wise."""
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


def mobius_handle(dims, U, Ls, b5, c5):
    return Handle(dims, U, Ls=Ls, M5=M5, mf=MF, mobius=True, b5=b5, c5=c5)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("dims,Ls,b5,c5", [((4, 4, 2, 4), 4, 1.5, 0.5), ((2, 6, 4, 2), 6, 2.0, 1.0),
                                          ((4, 2, 2, 4), 1, 1.25, 0.25), ((4, 4, 2, 4), 5, 1.0, 0.0)])
def test_mobius_dslash(prec, native, dims, Ls, b5, c5):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=1301)
    psi = inputs.gaussian_spinor(V, seed=2301, nrhs=Ls)
    H = mobius_handle(dims, U, Ls, b5, c5)
    try:
        for dag in (False, True):
            want = oracle.dwf_mobius_dslash(psi, U, dims, Ls, M5, MF, b5, c5, dagger=dag)
            x = dev(psi, prec)
            y = torch.empty_like(x)
            if native:
                nat = lqcd.LQ_NATIVE | prec
                xn, yn = native_buffer(H.h, prec, five_d=True), native_buffer(H.h, prec, five_d=True)
                lqcd.lq_convert(H.h, xn, nat, x, prec, five_d=True)
                lqcd.dwf_dslash_apply(H.h, yn, xn, nat, dag)
                lqcd.lq_convert(H.h, y, prec, yn, nat, five_d=True)
            else:
                lqcd.dwf_dslash_apply(H.h, y, x, prec, dag)
            check(host(y), want, prec)
    finally:
        H.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed_f32"])
def test_mobius_cg(mode):
    dims, Ls, b5, c5 = (4, 4, 4, 4), 6, 1.5, 0.5
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1302)
    eta = inputs.gaussian_spinor(V, seed=2302, nrhs=Ls)
    H = mobius_handle(dims, U, Ls, b5, c5)
    try:
        b = dev(oracle.dwf_mobius_dslash(eta, U, dims, Ls, M5, MF, b5, c5, dagger=True))
        x = torch.zeros_like(b)
        m = lqcd.LQ_CG_PLAIN if mode == "fp64" else lqcd.LQ_CG_MIXED
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, m, lqcd.LQ_F64, tol=1e-10, inner=lqcd.LQ_F32)
        rc, st = lqcd.cg_solve(H.h, x, b, cp)
        assert rc == 0 and st[0].true_rel_residual < 1e-10
        xs = host(x)
    finally:
        H.close()
    assert rel_err(oracle.dwf_mobius_dslash(xs, U, dims, Ls, M5, MF, b5, c5), eta) < 1e-7


def test_mobius_rejects_half_precision_and_a_singular_site_part():
    dims, Ls = (4, 4, 2, 4), 4
    V = int(np.prod(dims))
    H = mobius_handle(dims, inputs.gauge_field(dims, "unit"), Ls, 1.5, 0.5)
    try:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F16
        n = lqcd.lq_field_bytes(H.h, nat, five_d=True)
        a, b = (torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(2))
        with pytest.raises(lqcd.LqError):
            lqcd.dwf_dslash_apply(H.h, b, a, nat, False)
        with pytest.raises(lqcd.LqError):
            lqcd.dwf_schur_apply(H.h, b, a, nat, False)
        x = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device="cuda")
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, _ = lqcd.cg_solve(H.h, x, torch.ones_like(x), cp, check=False)
        assert rc == -1
    finally:
        H.close()
    # (4 - M5) b5 + 1 = 0: the site-local part M5_M has no inverse; D_M itself is still defined
    H = Handle(dims, inputs.gauge_field(dims, "unit"), Ls=Ls, M5=2.0, mf=MF, mobius=True, b5=-0.5, c5=0.5)
    try:
        xe = torch.zeros((Ls, V // 2, 4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(lqcd.LqError) as e:
            lqcd.dwf_schur_apply(H.h, torch.empty_like(xe), xe, lqcd.LQ_F64)
        assert e.value.status == -1
        x = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device="cuda")
        lqcd.dwf_dslash_apply(H.h, torch.empty_like(x), x, lqcd.LQ_F64, False)
    finally:
        H.close()


# ---------------------------------------------------------------- even-odd


EO_CASES = [((4, 4, 2, 4), 4, 1.5, 0.5), ((2, 6, 4, 2), 6, 2.0, 1.0), ((4, 2, 2, 4), 1, 1.25, 0.25),
            ((4, 4, 2, 4), 5, 1.0, 0.0), ((4, 4, 2, 4), 3, 0.8, -0.3)]


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
@pytest.mark.parametrize("native", [False, True])
@pytest.mark.parametrize("dims,Ls,b5,c5", EO_CASES)
def test_mobius_schur_apply(prec, native, dims, Ls, b5, c5):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=1311)
    x = inputs.gaussian_spinor(V // 2, seed=2311, nrhs=Ls)
    H = mobius_handle(dims, U, Ls, b5, c5)
    try:
        for dag in (False, True):
            want = oracle.dwf_mobius_schur(x, U, dims, Ls, M5, MF, b5, c5, dagger=dag)
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
    finally:
        H.close()


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (0.8, -0.3)])
def test_mobius_prepare_and_reconstruct(prec, b5, c5):
    dims, Ls = (4, 4, 2, 4), 5
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1312)
    eta = inputs.gaussian_spinor(V, seed=2312, nrhs=Ls)
    xe = inputs.gaussian_spinor(V // 2, seed=2313, nrhs=Ls)
    H = mobius_handle(dims, U, Ls, b5, c5)
    try:
        ed = dev(eta, prec)
        bh = torch.empty((Ls, V // 2, 4, 3), dtype=ed.dtype, device="cuda")
        lqcd.dwf_eo_prepare(H.h, bh, ed, prec)
        check(host(bh), oracle.dwf_mobius_eo_prepare(eta, U, dims, Ls, M5, MF, b5, c5), prec)
        psi = torch.empty_like(ed)
        lqcd.dwf_eo_reconstruct(H.h, psi, dev(xe, prec), ed, prec)
        check(host(psi), oracle.dwf_mobius_eo_reconstruct(xe, eta, U, dims, Ls, M5, MF, b5, c5), prec)
    finally:
        H.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed_f32"])
def test_mobius_eo_cg_solves_the_full_system(mode):
    """D_M psi = eta through the Schur complement: prepare the source, CG on
    Mhat^dag Mhat x_e = Mhat^dag bhat_e to 1e-10, reconstruct psi; psi must
    solve the full Moebius system (checked with the oracle's D_M)."""
    dims, Ls, b5, c5 = (4, 4, 4, 4), 6, 1.5, 0.5
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1314)
    eta = inputs.gaussian_spinor(V, seed=2314, nrhs=Ls)
    H = mobius_handle(dims, U, Ls, b5, c5)
    try:
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
    finally:
        H.close()
    # the normal-equation residual 1e-10 bounds |D_M psi - eta|/|eta| by about cond(Mhat) * 1e-10
    assert rel_err(oracle.dwf_mobius_dslash(p, U, dims, Ls, M5, MF, b5, c5), eta) < 1e-7


@pytest.mark.slow
def test_mobius_full_size_schur_f32():
    """16^4 x Ls 16 (the benchmark's domain-wall workload), FP32 native, both daggers."""
    dims, Ls, b5, c5 = (16, 16, 16, 16), 16, 1.5, 0.5
    U = inputs.gauge_field(dims, "smooth", seed=1004)
    x = inputs.gaussian_spinor(int(np.prod(dims)) // 2, seed=2004, nrhs=Ls)
    H = Handle(dims, U, Ls=Ls, M5=M5, mf=0.01, mobius=True, b5=b5, c5=c5)
    try:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        xn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_EVEN, Ls)
        yn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_EVEN, Ls)
        xd = dev(x, lqcd.LQ_F32)
        lqcd.lq_convert(H.h, xn, nat, xd, lqcd.LQ_F32, lqcd.LQ_EVEN, Ls)
        y = torch.empty_like(xd)
        for dag in (False, True):
            lqcd.dwf_schur_apply(H.h, yn, xn, nat, dag)
            lqcd.lq_convert(H.h, y, lqcd.LQ_F32, yn, nat, lqcd.LQ_EVEN, Ls)
            check(host(y), oracle.dwf_mobius_schur(x, U, dims, Ls, M5, 0.01, b5, c5, dagger=dag), lqcd.LQ_F32)
    finally:
        H.close()
