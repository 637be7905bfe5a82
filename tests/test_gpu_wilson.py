"""GPU parity: the CUDA Wilson / domain-wall operators against the FP64 oracle.

Tolerances (element-wise error relative to the largest reference element,
and norm-wise relative error), from the arithmetic of one hop: each output
component is a sum of ~30 rounded products/adds of inputs that were rounded
to the storage precision once.
  FP64:  1e-12 (the target); observed ~1e-15.
  FP32:  u = 2^-24; storage rounding + ~30-deep sums: 2e-6 norm-wise, 1e-5 element-wise.
  FP16:  per-site norm, u = 2^-11 on inputs, links and output: 2e-3 / 5e-3.
  BF16:  u = 2^-8: 1.5e-2 / 4e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, max_err, native_buffer, rel_err
from paper_2001_07557_gb300 import inputs
from paper_2001_07557_gb300 import lqcd

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQ_F64: (1e-12, 1e-12), lqcd.LQ_F32: (2e-6, 1e-5), lqcd.LQ_F16: (2e-3, 5e-3),
       lqcd.LQ_BF16: (1.5e-2, 4e-2)}

SHAPES = [((4, 4, 4, 4), (1, 1, 1, -1)), ((4, 6, 2, 8), (1, 1, 1, -1)), ((2, 2, 2, 2), (1, 1, 1, -1)),
          ((6, 4, 4, 2), (-1, 1, 1, 1)), ((8, 2, 6, 4), (1, -1, 1, -1))]


def check(got, want, prec):
    tn, te = TOL[prec]
    assert rel_err(got, want) <= tn, (rel_err(got, want), tn)
    assert max_err(got, want) <= te, (max_err(got, want), te)


def field(dims, kind="random", seed=1000):
    return inputs.gauge_field(dims, kind, seed=seed)


@pytest.mark.parametrize("dims,bc", SHAPES, ids=[str(s[0]) for s in SHAPES])
@pytest.mark.parametrize("dag", [False, True])
def test_full_wilson_f64_site_major(dims, bc, dag):
    V = int(np.prod(dims))
    U = field(dims, "random", 1000)
    psi = inputs.gaussian_spinor(V, seed=2000)
    want = oracle.wilson_dslash(psi, U, dims, 0.1, bc=bc, dagger=dag)
    with Handle(dims, U, mass=0.1, bc=bc) as H:
        x = dev(psi)
        y = torch.empty_like(x)
        (lqcd.dslash_dag_apply if dag else lqcd.dslash_apply)(H.h, y, x, lqcd.LQ_F64, lqcd.LQ_FULL)
        check(host(y), want, lqcd.LQ_F64)


@pytest.mark.parametrize("dims,bc", SHAPES[:4], ids=[str(s[0]) for s in SHAPES[:4]])
@pytest.mark.parametrize("dag", [False, True])
def test_eo_blocks_and_schur_f64(dims, bc, dag):
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1001)
    m = 0.05
    psi = inputs.gaussian_spinor(V, seed=2001)
    pe, po = inputs.to_half(psi, dims, 0), inputs.to_half(psi, dims, 1)
    with Handle(dims, U, mass=m, bc=bc) as H:
        fn = lqcd.dslash_dag_apply if dag else lqcd.dslash_apply
        for par, src in ((lqcd.LQ_EVEN, po), (lqcd.LQ_ODD, pe)):
            want = -0.5 * oracle.wilson_hop_eo(src, U, dims, par, bc=bc, dagger=dag)
            x = dev(src)
            y = torch.empty_like(x)
            fn(H.h, y, x, lqcd.LQ_F64, par)
            check(host(y), want, lqcd.LQ_F64)
        want = oracle.wilson_schur(pe, U, dims, m, bc=bc, dagger=dag)
        x = dev(pe)
        y = torch.empty_like(x)
        fn(H.h, y, x, lqcd.LQ_F64, lqcd.LQ_SCHUR_EVEN)
        check(host(y), want, lqcd.LQ_F64)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("r12", [False, True])
def test_native_precisions_full_and_schur(prec, r12):
    dims = (4, 6, 4, 8)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1002)
    m = 0.05
    psi = inputs.gaussian_spinor(V, seed=2002)
    pe = inputs.to_half(psi, dims, 0)
    with Handle(dims, U, mass=m, compress12=r12) as H:
        nat = lqcd.LQ_NATIVE | prec
        x = dev(psi)
        xn = native_buffer(H.h, prec)
        yn = native_buffer(H.h, prec)
        y = torch.empty_like(x)
        lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, lqcd.LQ_FULL)
        for dag in (False, True):
            fn = lqcd.dslash_dag_apply if dag else lqcd.dslash_apply
            fn(H.h, yn, xn, nat, lqcd.LQ_FULL)
            lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, lqcd.LQ_FULL)
            check(host(y), oracle.wilson_dslash(psi, U, dims, m, dagger=dag), prec)
        xe = dev(pe)
        xen = native_buffer(H.h, prec, lqcd.LQ_EVEN)
        yen = native_buffer(H.h, prec, lqcd.LQ_EVEN)
        ye = torch.empty_like(xe)
        lqcd.lq_convert(H.h, xen, nat, xe, lqcd.LQ_F64, lqcd.LQ_EVEN)
        lqcd.dslash_apply(H.h, yen, xen, nat, lqcd.LQ_SCHUR_EVEN)
        lqcd.lq_convert(H.h, ye, lqcd.LQ_F64, yen, nat, lqcd.LQ_EVEN)
        check(host(ye), oracle.wilson_schur(pe, U, dims, m), prec)


def test_f32_site_major_matches_native():
    dims = (4, 4, 6, 4)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1003)
    psi = inputs.gaussian_spinor(V, seed=2003)
    with Handle(dims, U, mass=0.2, U_prec=lqcd.LQ_F32) as H:
        x = dev(psi, lqcd.LQ_F32)
        y = torch.empty_like(x)
        lqcd.dslash_apply(H.h, y, x, lqcd.LQ_F32, lqcd.LQ_FULL)
        check(host(y), oracle.wilson_dslash(psi, U, dims, 0.2), lqcd.LQ_F32)
        xn = native_buffer(H.h, lqcd.LQ_F32)
        yn = native_buffer(H.h, lqcd.LQ_F32)
        y2 = torch.empty_like(x)
        lqcd.lq_convert(H.h, xn, lqcd.LQ_NATIVE | lqcd.LQ_F32, x, lqcd.LQ_F32)
        lqcd.dslash_apply(H.h, yn, xn, lqcd.LQ_NATIVE | lqcd.LQ_F32, lqcd.LQ_FULL)
        lqcd.lq_convert(H.h, y2, lqcd.LQ_F32, yn, lqcd.LQ_NATIVE | lqcd.LQ_F32)
        assert torch.equal(y, y2)


def test_conversion_round_trip_is_exact_in_f64():
    dims = (4, 2, 2, 6)
    V = int(np.prod(dims))
    U = field(dims, "unit")
    psi = inputs.gaussian_spinor(V, seed=5, nrhs=2)
    with Handle(dims, U) as H:
        x = dev(psi)
        n = native_buffer(H.h, lqcd.LQ_F64, nrhs=2)
        y = torch.empty_like(x)
        lqcd.lq_convert(H.h, n, lqcd.LQ_NATIVE | lqcd.LQ_F64, x, lqcd.LQ_F64, nrhs=2)
        lqcd.lq_convert(H.h, y, lqcd.LQ_F64, n, lqcd.LQ_NATIVE | lqcd.LQ_F64, nrhs=2)
        assert torch.equal(x, y)


@pytest.mark.parametrize("nrhs", [2, 5])
def test_multi_rhs_f64(nrhs):
    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    U = field(dims, "random", 1004)
    psi = inputs.gaussian_spinor(V, seed=2004, nrhs=nrhs)
    with Handle(dims, U, mass=0.1) as H:
        x = dev(psi)
        y = torch.empty_like(x)
        lqcd.dslash_apply(H.h, y, x, lqcd.LQ_F64, lqcd.LQ_FULL, nrhs=nrhs)
        check(host(y), oracle.wilson_dslash(psi, U, dims, 0.1), lqcd.LQ_F64)
        pe = inputs.to_half(psi, dims, 0)
        xe = dev(pe)
        ye = torch.empty_like(xe)
        lqcd.dslash_apply(H.h, ye, xe, lqcd.LQ_F64, lqcd.LQ_SCHUR_EVEN, nrhs=nrhs)
        check(host(ye), oracle.wilson_schur(pe, U, dims, 0.1), lqcd.LQ_F64)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16])
@pytest.mark.parametrize("dag", [False, True])
def test_domain_wall(prec, dag):
    dims = (4, 4, 2, 4)
    Ls, M5, mf = 6, 1.8, 0.01
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1005)
    psi = inputs.gaussian_spinor(V, seed=2005, nrhs=Ls)
    want = oracle.dwf_dslash(psi, U, dims, Ls, M5, mf, dagger=dag)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=mf) as H:
        x = dev(psi)
        y = torch.empty_like(x)
        if prec == lqcd.LQ_F64:
            lqcd.dwf_dslash_apply(H.h, y, x, lqcd.LQ_F64, dag)
        else:
            nat = lqcd.LQ_NATIVE | prec
            xn = native_buffer(H.h, prec, five_d=True)
            yn = native_buffer(H.h, prec, five_d=True)
            lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, five_d=True)
            lqcd.dwf_dslash_apply(H.h, yn, xn, nat, dag)
            lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, five_d=True)
        check(host(y), want, prec)


def test_domain_wall_ls1_reduces_to_wilson():
    dims = (4, 2, 4, 2)
    V = int(np.prod(dims))
    U = field(dims, "random", 1006)
    psi = inputs.gaussian_spinor(V, seed=2006)
    with Handle(dims, U, Ls=1, M5=1.8, mf=0.01) as H:
        x = dev(psi[None])
        y = torch.empty_like(x)
        lqcd.dwf_dslash_apply(H.h, y, x, lqcd.LQ_F64, False)
        check(host(y)[0], oracle.wilson_dslash(psi, U, dims, 1 - 1.8 + 0.01), lqcd.LQ_F64)


def test_error_paths():
    dims = (4, 4, 4, 4)
    U = field(dims, "unit")
    with Handle(dims, U) as H:
        x = dev(inputs.gaussian_spinor(256, seed=1))
        y = torch.empty_like(x)
        L = lqcd.lib()
        st = torch.cuda.current_stream().cuda_stream
        assert L.dslash_apply(H.h, y.data_ptr() + 8, x.data_ptr(), 0, -1, 1, st) == -2   # misaligned
        assert L.dslash_apply(H.h, x.data_ptr(), x.data_ptr(), 0, -1, 1, st) == -1       # aliasing
        assert L.dslash_apply(H.h, y.data_ptr(), x.data_ptr(), 7, -1, 1, st) == -1       # bad format
        assert L.dslash_apply(H.h, y.data_ptr(), x.data_ptr(), 0, 3, 1, st) == -1        # bad parity
        assert L.dslash_apply(H.h, y.data_ptr(), x.data_ptr(), 0, -1, 0, st) == -1       # no rhs
        assert L.dslash_apply(H.h, y.data_ptr(), x.data_ptr(), lqcd.LQ_F16, -1, 1, st) == -1  # f16 site-major
        assert L.dwf_dslash_apply(H.h, y.data_ptr(), x.data_ptr(), 0, 0, st) == -1      # Ls = 0
    Ud = dev(U)
    for bad in [lqcd.make_params((4, 4, 3, 4)), lqcd.make_params((4, 4, 4, 4), r=0.5),
                lqcd.make_params((4, 4, 4, 4), bc=(1, 1, 1, 2)), lqcd.make_params((0, 4, 4, 4))]:
        with pytest.raises(lqcd.LqError):
            lqcd.lq_create(bad, Ud)


@pytest.mark.slow
def test_full_size_32x4_eo_f32_native_sampled():
    """32^4, smooth links, m = 0.01: the even-odd FP32 hop in the launch
    configuration the benchmark times, against the oracle on the whole lattice."""
    dims = (32, 32, 32, 32)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1002)
    psi = inputs.gaussian_spinor(V // 2, seed=2002)
    rng = np.random.default_rng(0)
    sample = rng.choice(V // 2, 4096, replace=False)
    with Handle(dims, U, mass=0.01) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        x = dev(psi)
        xn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_ODD)
        yn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_EVEN)
        y = torch.empty_like(x)
        lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, lqcd.LQ_ODD)
        lqcd.dslash_apply(H.h, yn, xn, nat, lqcd.LQ_EVEN)
        lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, lqcd.LQ_EVEN)
        got = host(y)[sample]
    want = (-0.5 * oracle.wilson_hop_eo(psi, U, dims, 0))[sample]
    check(got, want, lqcd.LQ_F32)


@pytest.mark.slow
def test_full_size_bench_step_fp16_normal_operator():
    """The benchmark's step in its launch configuration: 32^4, smooth links,
    m = 0.01, FP16 storage with per-site norms, 18-real links, Mhat^dag Mhat on
    a Gaussian even field -- against the oracle on the whole lattice."""
    dims = (32, 32, 32, 32)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1002)
    psi = inputs.gaussian_spinor(V // 2, seed=2002)
    with Handle(dims, U, mass=0.01) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F16
        x = dev(psi)
        xn, yn, zn = (native_buffer(H.h, lqcd.LQ_F16, lqcd.LQ_EVEN) for _ in range(3))
        lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, lqcd.LQ_EVEN)
        lqcd.dslash_apply(H.h, yn, xn, nat, lqcd.LQ_SCHUR_EVEN)
        lqcd.dslash_dag_apply(H.h, zn, yn, nat, lqcd.LQ_SCHUR_EVEN)
        z = torch.empty_like(x)
        lqcd.lq_convert(H.h, z, lqcd.LQ_F64, zn, nat, lqcd.LQ_EVEN)
        got = host(z)
    want = oracle.apply_normal(oracle.OP_WILSON_EO, psi, U, oracle.params(dims, mass=0.01))
    # two FP16 operator applications: twice the single-hop tolerance
    assert rel_err(got, want) < 4e-3
    assert max_err(got, want) < 1e-2


@pytest.mark.slow
def test_full_size_multi_rhs_fp16_point_sources():
    """24^3x48, smooth links, m = 0.02, 12 point sources, FP16 full-lattice D in
    one 12-right-hand-side launch; three of the twelve checked against the oracle."""
    dims = (24, 24, 24, 48)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1003)
    src = inputs.point_sources(V)
    with Handle(dims, U, mass=0.02) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F16
        x = dev(src)
        xn = native_buffer(H.h, lqcd.LQ_F16, lqcd.LQ_FULL, 12)
        yn = native_buffer(H.h, lqcd.LQ_F16, lqcd.LQ_FULL, 12)
        lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, lqcd.LQ_FULL, 12)
        lqcd.dslash_apply(H.h, yn, xn, nat, lqcd.LQ_FULL, nrhs=12)
        y = torch.empty_like(x)
        lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, lqcd.LQ_FULL, 12)
        got = host(y)
    for k in (0, 5, 11):
        check(got[k], oracle.wilson_dslash(src[k], U, dims, 0.02), lqcd.LQ_F16)


@pytest.mark.slow
def test_full_size_multi_rhs_fp32_point_sources():
    """24^3x48, smooth links, m = 0.02, the 12 point sources stored as FP32 spinors
    (the multi-right-hand-side workload's own precision), 18-real links: the full-lattice
    D of all twelve in one launch, in the launch configuration the bench times, checked
    element by element against the oracle for four of the sources (FP32 tolerance)."""
    dims = (24, 24, 24, 48)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1003)
    src = inputs.point_sources(V)
    with Handle(dims, U, mass=0.02) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        x = dev(src, lqcd.LQ_F32)
        xn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_FULL, 12)
        yn = native_buffer(H.h, lqcd.LQ_F32, lqcd.LQ_FULL, 12)
        lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F32, lqcd.LQ_FULL, 12)
        lqcd.dslash_apply(H.h, yn, xn, nat, lqcd.LQ_FULL, nrhs=12)
        y = torch.empty_like(x)
        lqcd.lq_convert(H.h, y, lqcd.LQ_F32, yn, nat, lqcd.LQ_FULL, 12)
        got = host(y)
    for k in (0, 4, 7, 11):
        check(got[k], oracle.wilson_dslash(src[k], U, dims, 0.02), lqcd.LQ_F32)


@pytest.mark.slow
@pytest.mark.parametrize("prec", [lqcd.LQ_F32, lqcd.LQ_F16])
def test_full_size_domain_wall(prec):
    """16^4 x Ls = 16, M5 = 1.8, mf = 0.01, smooth links, Gaussian 5-d field,
    18-real links: the benchmark's domain-wall launch against the oracle."""
    dims = (16, 16, 16, 16)
    Ls = 16
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1004)
    psi = inputs.gaussian_spinor(V, seed=2004, nrhs=Ls)
    with Handle(dims, U, Ls=Ls, M5=1.8, mf=0.01) as H:
        nat = lqcd.LQ_NATIVE | prec
        x = dev(psi)
        xn = native_buffer(H.h, prec, five_d=True)
        yn = native_buffer(H.h, prec, five_d=True)
        lqcd.lq_convert(H.h, xn, nat, x, lqcd.LQ_F64, five_d=True)
        lqcd.dwf_dslash_apply(H.h, yn, xn, nat, False)
        y = torch.empty_like(x)
        lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, five_d=True)
        got = host(y)
    check(got, oracle.dwf_dslash(psi, U, dims, Ls, 1.8, 0.01), prec)


def test_convert_reads_and_writes_pinned_host_memory():
    """lq_convert with a pinned host source and destination: the conversion
    kernels address host memory directly; the round trip is exact."""
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    psi = inputs.gaussian_spinor(V, seed=2401)
    with Handle(dims, field(dims, "unit")) as H:
        hx = torch.from_numpy(psi.astype(np.complex64)).pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        n = native_buffer(H.h, lqcd.LQ_F32)
        lqcd.lq_convert(H.h, n, lqcd.LQ_NATIVE | lqcd.LQ_F32, hx, lqcd.LQ_F32)
        lqcd.lq_convert(H.h, hy, lqcd.LQ_F32, n, lqcd.LQ_NATIVE | lqcd.LQ_F32)
        torch.cuda.synchronize()
        assert torch.equal(hy, hx)


SHARED_SHAPES = [((4, 6, 2, 8), (1, 1, 1, -1)),   # Vh = 192: three 64-site tiles (an odd count)
                 ((8, 2, 6, 4), (1, -1, 1, -1)),  # Vh = 192, antiperiodic y
                 ((6, 4, 4, 2), (-1, 1, 1, 1))]   # Vh = 96: one full and one ragged tile


@pytest.mark.parametrize("dims,bc", SHARED_SHAPES, ids=[str(s[0]) for s in SHARED_SHAPES])
@pytest.mark.parametrize("prec,r12", [(lqcd.LQ_F32, False), (lqcd.LQ_F32, True), (lqcd.LQ_F16, False),
                                      (lqcd.LQ_F16, True), (lqcd.LQ_BF16, False)])
@pytest.mark.parametrize("dag", [False, True])
def test_multi_rhs_launch_equals_single_launches_bit_for_bit(dims, bc, prec, r12, dag):
    """A launch of several right-hand sides (FP32: the kernel whose blocks share each
    link between them) gives every right-hand side bit for bit what a launch of its own
    gives, for the full operator, an even-odd block and the Schur complement; 5
    right-hand sides (groups with one and two of them) and 9."""
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1001)
    nat = lqcd.LQ_NATIVE | prec
    fn = lqcd.dslash_dag_apply if dag else lqcd.dslash_apply
    with Handle(dims, U, mass=0.05, bc=bc, compress12=r12) as H:
        for nrhs in (5, 9):
            psi = inputs.gaussian_spinor(V, seed=2100 + nrhs, nrhs=nrhs)
            for parity, sub_in, sub_out in ((lqcd.LQ_FULL, lqcd.LQ_FULL, lqcd.LQ_FULL),
                                            (lqcd.LQ_EVEN, lqcd.LQ_ODD, lqcd.LQ_EVEN),
                                            (lqcd.LQ_SCHUR_EVEN, lqcd.LQ_EVEN, lqcd.LQ_EVEN)):
                src = psi if sub_in == lqcd.LQ_FULL else np.stack([inputs.to_half(q, dims, sub_in) for q in psi])
                xn = native_buffer(H.h, prec, sub_in, nrhs)
                yn = native_buffer(H.h, prec, sub_out, nrhs)
                lqcd.lq_convert(H.h, xn, nat, dev(src), lqcd.LQ_F64, sub_in, nrhs)
                fn(H.h, yn, xn, nat, parity, nrhs=nrhs)
                one_in = xn.numel() // nrhs
                one_out = yn.numel() // nrhs
                for k in range(nrhs):
                    yk = native_buffer(H.h, prec, sub_out, 1)
                    fn(H.h, yk, xn[k * one_in:(k + 1) * one_in], nat, parity, nrhs=1)
                    assert torch.equal(yk, yn[k * one_out:(k + 1) * one_out]), (nrhs, parity, k)


@pytest.mark.parametrize("prec", [lqcd.LQ_F32, lqcd.LQ_F16])
def test_domain_wall_slices_match_their_oracle_on_odd_tile_counts(prec):
    """Domain wall on 4x6x2x8 (three 64-site tiles per parity) with Ls = 3 and 7:
    the launch over all slices against the oracle, both daggers."""
    dims = (4, 6, 2, 8)
    V = int(np.prod(dims))
    U = field(dims, "smooth", 1004)
    for Ls in (3, 7):
        psi = inputs.gaussian_spinor(V, seed=2300 + Ls, nrhs=Ls)
        with Handle(dims, U, Ls=Ls, M5=1.8, mf=0.01) as H:
            nat = lqcd.LQ_NATIVE | prec
            for dag in (False, True):
                xn = native_buffer(H.h, prec, five_d=True)
                yn = native_buffer(H.h, prec, five_d=True)
                lqcd.lq_convert(H.h, xn, nat, dev(psi), lqcd.LQ_F64, five_d=True)
                lqcd.dwf_dslash_apply(H.h, yn, xn, nat, dag)
                y = torch.empty_like(dev(psi))
                lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, five_d=True)
                check(host(y), oracle.dwf_dslash(psi, U, dims, Ls, 1.8, 0.01, dagger=dag), prec)
