"""GPU parity: the tensor-core multi-right-hand-side hop (lq_set_hop_kernel
LQ_HOP_TENSOR_CORES; FP16/BF16 storage, at least 8 right-hand sides, one m16n8k8
MMA per site, direction and group of 8) against the FP64 oracle, and against
the CUDA-core hop of the same handle.

Tolerances are those of the FP16/BF16 hop (tests/test_gpu_wilson.py): the MMA
multiplies the same 16-bit inputs and accumulates in FP32, so only the order
of the FP32 sums differs from the CUDA-core kernel.  Lattices with V/2 not a
multiple of the 32-site tile exercise the ragged last tile; 12 and 17
right-hand sides a partly filled last group.
"""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, max_err, native_buffer, rel_err
from paper_2001_07557_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQ_F16: (2e-3, 5e-3), lqcd.LQ_BF16: (1.5e-2, 4e-2)}


def check(got, want, prec):
    tn, te = TOL[prec]
    assert rel_err(got, want) <= tn, (rel_err(got, want), tn)
    assert max_err(got, want) <= te, (max_err(got, want), te)


def apply(H, prec, psi, parity, nrhs, dag, kind):
    """The operator selected by `parity` on nrhs site-major FP64 fields through native storage."""
    lqcd.lq_set_hop_kernel(H.h, kind)
    nat = lqcd.LQ_NATIVE | prec
    sub = lqcd.LQ_FULL if parity == lqcd.LQ_FULL else lqcd.LQ_EVEN
    x = dev(psi)
    xn, yn = native_buffer(H.h, prec, sub, nrhs), native_buffer(H.h, prec, sub, nrhs)
    lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, sub, nrhs)
    (lqcd.dslash_dag_apply if dag else lqcd.dslash_apply)(H.h, yn, xn, nat, parity, nrhs)
    y = torch.empty_like(x)
    lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, sub, nrhs)
    return host(y)


@pytest.mark.parametrize("prec", [lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("dims,bc,nrhs", [((4, 2, 2, 6), (1, 1, 1, -1), 8), ((6, 4, 2, 4), (1, 1, 1, -1), 12),
                                          ((4, 4, 4, 4), (-1, 1, 1, -1), 17), ((8, 2, 6, 4), (1, -1, 1, -1), 16)])
def test_full_operator_matches_oracle_and_cuda_cores(prec, dims, bc, nrhs):
    V = int(np.prod(dims))
    m = 0.05
    U = inputs.gauge_field(dims, "random", seed=1401)
    psi = inputs.gaussian_spinor(V, seed=2401, nrhs=nrhs)
    with Handle(dims, U, mass=m, bc=bc) as H:
        for dag in (False, True):
            tc = apply(H, prec, psi, lqcd.LQ_FULL, nrhs, dag, lqcd.LQ_HOP_TENSOR_CORES)
            cc = apply(H, prec, psi, lqcd.LQ_FULL, nrhs, dag, lqcd.LQ_HOP_CUDA_CORES)
            for k in range(nrhs):
                want = oracle.wilson_dslash(psi[k], U, dims, m, bc=bc, dagger=dag)
                check(tc[k], want, prec)
                check(cc[k], want, prec)


@pytest.mark.parametrize("prec", [lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("parity", [lqcd.LQ_SCHUR_EVEN, lqcd.LQ_EVEN, lqcd.LQ_ODD])
def test_even_odd_blocks_and_schur(prec, parity):
    """One-parity launches: the plain hop between parities (LQ_EVEN / LQ_ODD give
    D's off-diagonal block -1/2 H) and the Schur complement (two launches, the
    second with the diagonal input), 12 right-hand sides."""
    dims, nrhs, m = (6, 4, 2, 4), 12, 0.05
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1402)
    full = inputs.gaussian_spinor(V, seed=2402, nrhs=nrhs)
    src_par = 1 - parity if parity in (lqcd.LQ_EVEN, lqcd.LQ_ODD) else 0
    half = np.stack([inputs.to_half(full[k], dims, src_par) for k in range(nrhs)])
    with Handle(dims, U, mass=m) as H:
        for dag in (False, True):
            if parity == lqcd.LQ_SCHUR_EVEN:
                got = apply(H, prec, half, parity, nrhs, dag, lqcd.LQ_HOP_TENSOR_CORES)
                for k in range(nrhs):
                    check(got[k], oracle.wilson_schur(half[k], U, dims, m, dagger=dag), prec)
            else:
                lqcd.lq_set_hop_kernel(H.h, lqcd.LQ_HOP_TENSOR_CORES)
                nat = lqcd.LQ_NATIVE | prec
                x = dev(half)
                xn, yn = (native_buffer(H.h, prec, lqcd.LQ_EVEN, nrhs) for _ in range(2))
                lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, src_par, nrhs)
                (lqcd.dslash_dag_apply if dag else lqcd.dslash_apply)(H.h, yn, xn, nat, parity, nrhs)
                y = torch.empty_like(x)
                lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, parity, nrhs)
                got = host(y)
                for k in range(nrhs):
                    want = -0.5 * oracle.wilson_hop_eo(half[k], U, dims, parity, dagger=dag)
                    check(got[k], want, prec)


def test_batched_mixed_cg_with_a_zero_source():
    """Batched mixed CG (FP16 inner) on 12 right-hand sides: the inner hops run
    on the tensor cores with the fused norm; a zero source is finished before
    the first iteration, so its rows are skipped in every launch and its
    solution stays zero.  The other 11 solve D x = source to 1e-10."""
    dims, m = (4, 4, 4, 8), 0.05
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1403)
    src = inputs.point_sources(V)
    src[5] = 0
    b = np.stack([oracle.wilson_dslash(src[k], U, dims, m, dagger=True) for k in range(12)])
    with Handle(dims, U, mass=m) as H:
        lqcd.lq_set_hop_kernel(H.h, lqcd.LQ_HOP_TENSOR_CORES)
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=12, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    assert not np.any(xg[5])
    for k in range(12):
        if k == 5:
            continue
        assert st[k].true_rel_residual < 1e-10
        assert rel_err(oracle.wilson_dslash(xg[k], U, dims, m), src[k]) < 1e-8


def test_set_hop_kernel_rejects_unknown_kinds():
    dims = (4, 4, 2, 4)
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        with pytest.raises(lqcd.LqError):
            lqcd.lq_set_hop_kernel(H.h, 2)


@pytest.mark.parametrize("prec", [lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("dims,Ls", [((4, 4, 2, 6), 8), ((4, 6, 2, 4), 12), ((4, 4, 4, 4), 16)])
def test_domain_wall_matches_oracle_and_cuda_cores(prec, dims, Ls):
    """The domain-wall operator with its Ls slices as the tensor-core kernel's right-hand
    sides (Ls = 12: a partly filled second group), both daggers, against the oracle's
    D_dw and the CUDA-core hop of the same handle."""
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1402)
    psi = inputs.gaussian_spinor(V, seed=2402, nrhs=Ls)
    nat = lqcd.LQ_NATIVE | prec
    with Handle(dims, U, Ls=Ls, M5=1.8, mf=0.01) as H:
        for dag in (False, True):
            out = {}
            for kind in (lqcd.LQ_HOP_TENSOR_CORES, lqcd.LQ_HOP_CUDA_CORES):
                lqcd.lq_set_hop_kernel(H.h, kind)
                xn, yn = native_buffer(H.h, prec, five_d=True), native_buffer(H.h, prec, five_d=True)
                lqcd.lq_convert(H.h, xn, nat, dev(psi), lqcd.LQ_F64, five_d=True)
                lqcd.dwf_dslash_apply(H.h, yn, xn, nat, dag)
                y = torch.empty_like(dev(psi))
                lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, five_d=True)
                out[kind] = host(y)
            want = oracle.dwf_dslash(psi, U, dims, Ls, 1.8, 0.01, dagger=dag)
            check(out[lqcd.LQ_HOP_TENSOR_CORES], want, prec)
            check(out[lqcd.LQ_HOP_CUDA_CORES], want, prec)


def test_domain_wall_mixed_cg_on_the_tensor_cores():
    """CG on D_dw^dag D_dw (Ls = 8) refined in FP64 around FP16 inner solves whose operator
    runs on the tensor cores, with the fused norm of the 5-d system in the kernel's slots:
    the oracle's D_dw maps the solution back to eta."""
    dims, Ls = (4, 4, 4, 4), 8
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1403)
    eta = inputs.gaussian_spinor(V, seed=2403, nrhs=Ls)
    prm = oracle.params(dims, Ls=Ls, M5=1.8, mf=0.01)
    b = oracle.apply_op(oracle.OP_DWF, eta, U, prm, dagger=True)
    with Handle(dims, U, Ls=Ls, M5=1.8, mf=0.01) as H:
        lqcd.lq_set_hop_kernel(H.h, lqcd.LQ_HOP_TENSOR_CORES)
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10, maxiter=40000,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0 and st[0].true_rel_residual < 1e-10
    assert rel_err(oracle.apply_op(oracle.OP_DWF, xg, U, prm), eta) < 1e-8
