"""GPU CG solvers against the FP64 oracle.

FP64 CG: the solution must satisfy the FP64 true residual |b - A x|/|b| < 1e-12
(the solver restarts from its iterate until its true residual, not only its
recursive one, is below tol) and agree with the oracle's dense-LU solution
within kappa(A) * tol.  Mixed precision: true residual <= the
requested 1e-10 and agreement with the oracle's FP64 CG within kappa * tol.
"""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, rel_err
from paper_2001_07557_gb300 import inputs
from paper_2001_07557_gb300 import lqcd

pytestmark = pytest.mark.gpu


def dense_D(U, dims, m):
    V = int(np.prod(dims))
    n = V * 12
    M = np.empty((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for k in range(n):
        e[:] = 0
        e[k] = 1
        M[:, k] = oracle.wilson_dslash(e.reshape(V, 4, 3), U, dims, m).ravel()
    return M


def test_c1_fp64_cg_matches_dense_lu():
    """4^4, random SU(3), m = 0.1, CG on D^dag D x = D^dag eta to 1e-12."""
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "random", seed=1000)
    eta = inputs.gaussian_spinor(256, seed=2000)
    D = dense_D(U, dims, 0.1)
    x_lu = np.linalg.solve(D, eta.ravel()).reshape(256, 4, 3)
    sv = np.linalg.svd(D, compute_uv=False)
    kappa = (sv[0] / sv[-1]) ** 2
    b = oracle.wilson_dslash(eta, U, dims, 0.1, dagger=True)
    # the FP64 CG iterates to tol / 2 so that its true residual lands below tol: the oracle's CG to
    # the same recursive target takes the same number of iterations
    _, it_or, _, _ = oracle.cg(oracle.OP_WILSON, b, U, oracle.params(dims, mass=0.1), 0.5e-12)
    with Handle(dims, U, mass=0.1) as H:
        x = torch.zeros(256, 4, 3, dtype=torch.complex128, device="cuda")
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, tol=1e-12)
        rc, st = lqcd.cg_solve(H.h, x, dev(b), cp)
        xg = host(x)
    assert rc == 0 and st[0].status == 0
    assert st[0].true_rel_residual < 1e-12
    assert abs(st[0].iters - it_or) <= 2
    assert rel_err(xg, x_lu) < 1e-12 * kappa


@pytest.mark.parametrize("fmt", [lqcd.LQ_F64, lqcd.LQ_NATIVE | lqcd.LQ_F64])
def test_eo_fp64_cg(fmt):
    dims = (8, 8, 8, 8)
    V = 8 ** 4
    m = 0.05
    U = inputs.gauge_field(dims, "smooth", seed=1001)
    be = inputs.gaussian_spinor(V // 2, seed=2001)
    prm = oracle.params(dims, mass=m)
    x_or, it_or, _, rc_or = oracle.cg(oracle.OP_WILSON_EO, be, U, prm, 1e-10)
    assert rc_or == oracle.OK
    with Handle(dims, U, mass=m) as H:
        bd = dev(be)
        xd = torch.zeros_like(bd)
        if fmt & lqcd.LQ_NATIVE:
            n = lqcd.lq_field_bytes(H.h, fmt, lqcd.LQ_EVEN)
            bn = torch.empty(n, dtype=torch.uint8, device="cuda")
            xn = torch.empty(n, dtype=torch.uint8, device="cuda")
            lqcd.lq_convert(H.h, bn, fmt, bd, lqcd.LQ_F64, lqcd.LQ_EVEN)
            cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, fmt, tol=1e-10)
            rc, st = lqcd.cg_solve(H.h, xn, bn, cp)
            lqcd.lq_convert(H.h, xd, lqcd.LQ_F64, xn, fmt, lqcd.LQ_EVEN)
        else:
            cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, fmt, tol=1e-10)
            rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    assert st[0].true_rel_residual < 1e-10
    assert abs(st[0].iters - it_or) <= 3
    assert rel_err(xg, x_or) < 1e-7


@pytest.mark.parametrize("inner", [lqcd.LQ_F32, lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("r12", [False, True])
def test_mixed_eo_reaches_1e10(inner, r12):
    dims = (8, 8, 8, 16)
    V = int(np.prod(dims))
    m = 0.02
    U = inputs.gauge_field(dims, "smooth", seed=1002)
    be = inputs.gaussian_spinor(V // 2, seed=2002)
    x_or, _, _, _ = oracle.cg(oracle.OP_WILSON_EO, be, U, oracle.params(dims, mass=m), 1e-12)
    with Handle(dims, U, mass=m, compress12=r12) as H:
        bd = dev(be)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10,
                                 inner=inner)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0, lqcd.STATUS[rc]
    assert st[0].true_rel_residual < 1e-10
    assert st[0].outer_iters >= 1
    assert rel_err(xg, x_or) < 1e-7


def test_mixed_multi_rhs_point_sources_full_operator():
    """Four of the 12 point sources, full-lattice D^dag D, batched mixed CG (FP16 inner)."""
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    m = 0.05
    U = inputs.gauge_field(dims, "smooth", seed=1003)
    src = inputs.point_sources(V)[[0, 4, 7, 11]]
    b = oracle.wilson_dslash(src, U, dims, m, dagger=True)
    with Handle(dims, U, mass=m) as H:
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=4, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    for k in range(4):
        assert st[k].true_rel_residual < 1e-10
        # D x = source
        assert rel_err(oracle.wilson_dslash(xg[k], U, dims, m), src[k]) < 1e-8


def test_fp32_plain_cg():
    dims = (4, 4, 8, 8)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1004)
    be = inputs.gaussian_spinor(V // 2, seed=2004)
    with Handle(dims, U, mass=0.1) as H:
        bd = dev(be, lqcd.LQ_F32)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F32, tol=1e-5)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
    assert rc == 0
    assert st[0].true_rel_residual < 5e-5


def test_dwf_cg_fp32_then_mixed_refinement():
    """Domain wall: CG on D_dw^dag D_dw in FP32 to 1e-8 is out of FP32's reach,
    so the mixed solver (FP32 inner) refines in FP64 to 1e-10."""
    dims = (4, 4, 4, 4)
    Ls, M5, mf = 8, 1.8, 0.01
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1005)
    eta = inputs.gaussian_spinor(V, seed=2005, nrhs=Ls)
    prm = oracle.params(dims, Ls=Ls, M5=M5, mf=mf)
    b = oracle.apply_op(oracle.OP_DWF, eta, U, prm, dagger=True)
    with Handle(dims, U, Ls=Ls, M5=M5, mf=mf) as H:
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10,
                                 inner=lqcd.LQ_F32, inner_tol=1e-6)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    assert st[0].true_rel_residual < 1e-10
    assert rel_err(oracle.apply_op(oracle.OP_DWF, xg, U, prm), eta) < 1e-8


def test_restart_from_guess_and_maxiter():
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "random", seed=1000)
    b = inputs.gaussian_spinor(256, seed=2007)
    with Handle(dims, U, mass=0.1) as H:
        bd = dev(b)
        x = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, tol=1e-12, maxiter=3)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp, check=False)
        assert rc == -5 and st[0].status == -5 and st[0].iters == 3
        # restart from the 3-iteration iterate
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, tol=1e-12,
                                 x0_is_guess=True)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp)
        assert rc == 0 and st[0].true_rel_residual < 1e-12
        # a guess that already meets the tolerance needs no iterations
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, tol=1e-10,
                                 x0_is_guess=True)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp)
        assert rc == 0 and st[0].iters == 0 and st[0].true_rel_residual < 1e-12


def test_nan_source_is_reported():
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "unit")
    b = inputs.gaussian_spinor(256, seed=1)
    b[17, 2, 1] = np.nan
    with Handle(dims, U, mass=0.1) as H:
        bd = dev(b)
        x = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, tol=1e-10)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp, check=False)
        assert rc == -8 and st[0].status == -8
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.cg_solve(H.h, x, bd, cp, check=False)
        assert rc == -8


def test_block_cg_twelve_point_sources():
    """12 point sources (one per spin-colour at the origin), block CG on D^dag D
    inside the FP64 defect correction, to 1e-10; each column solves D x = source."""
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    m = 0.05
    U = inputs.gauge_field(dims, "smooth", seed=1003)
    src = inputs.point_sources(V)
    b = oracle.wilson_dslash(src, U, dims, m, dagger=True)
    with Handle(dims, U, mass=m) as H:
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_BLOCK, lqcd.LQ_F64, nrhs=12, tol=1e-10)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
        cpb = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=12, tol=1e-10,
                                  inner=lqcd.LQ_F32, inner_tol=1e-5)
        rcb, stb = lqcd.cg_solve(H.h, torch.zeros_like(bd), bd, cpb)
    assert rc == 0
    for k in range(12):
        assert st[k].true_rel_residual < 1e-10
        assert rel_err(oracle.wilson_dslash(xg[k], U, dims, m), src[k]) < 1e-8
    # the block Krylov space needs fewer operator applications than 12 independent solves
    assert max(s.iters for s in st) < max(s.iters for s in stb)


def test_block_cg_even_odd_gaussian():
    dims = (4, 4, 8, 8)
    V = int(np.prod(dims))
    m = 0.05
    U = inputs.gauge_field(dims, "smooth", seed=1006)
    be = inputs.gaussian_spinor(V // 2, seed=2006, nrhs=5)
    prm = oracle.params(dims, mass=m)
    with Handle(dims, U, mass=m) as H:
        bd = dev(be)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_BLOCK, lqcd.LQ_F64, nrhs=5, tol=1e-10)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    for k in range(5):
        assert st[k].true_rel_residual < 1e-10
        x_or, _, _, _ = oracle.cg(oracle.OP_WILSON_EO, be[k], U, prm, 1e-12)
        assert rel_err(xg[k], x_or) < 1e-7


@pytest.mark.parametrize("op", [lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_OP_WILSON_NORMAL])
def test_block_cg_repeats_bit_for_bit(op):
    """The Gram of K P runs on a second stream beside the K^dag stage of the operator; the order of
    the two streams' work is fixed by events, so repeated solves give the same bits (a missing
    dependency would let the Gram read a half-written K P, or overwrite the sums the other stream
    reads, and change the iterates).  Checked against the oracle's operator once."""
    dims = (12, 12, 12, 16)
    V = int(np.prod(dims))
    m = 0.05
    U = inputs.gauge_field(dims, "smooth", seed=1009)
    n = V // 2 if op == lqcd.LQ_OP_WILSON_EO_NORMAL else V
    b = inputs.gaussian_spinor(n, seed=2009, nrhs=12)
    with Handle(dims, U, mass=m) as H:
        bd = dev(b)
        cp = lqcd.make_cg_params(op, lqcd.LQ_CG_BLOCK, lqcd.LQ_F64, nrhs=12, tol=1e-10)
        runs = []
        for _ in range(3):
            xd = torch.zeros_like(bd)
            rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
            assert rc == 0
            runs.append((xd, [s_.iters for s_ in st], [s_.true_rel_residual for s_ in st]))
    for xd, iters, res in runs[1:]:
        assert torch.equal(xd, runs[0][0]) and iters == runs[0][1] and res == runs[0][2]
    assert max(runs[0][2]) < 1e-10
    oop = oracle.OP_WILSON_EO if op == lqcd.LQ_OP_WILSON_EO_NORMAL else oracle.OP_WILSON
    xg = host(runs[0][0])
    prm = oracle.params(dims, mass=m)
    assert rel_err(oracle.apply_normal(oop, xg[5], U, prm), b[5]) < 1e-9


@pytest.mark.parametrize("nrhs", [1, 3, 4, 9, 16])
def test_block_cg_ragged_tiles_and_sizes(nrhs):
    """Block sizes 1, 3 (odd: one warp owns a single column), 4 (one whole
    group of the Gram kernel), 9 (a last group of one column: every kind of
    Gram block, diagonal or not, whole or ragged) and 16 (the largest) on a
    lattice whose field length is not a whole number of tiles."""
    dims = (6, 2, 2, 6)
    V = int(np.prod(dims))
    m = 0.1
    U = inputs.gauge_field(dims, "random", seed=1007)
    b = inputs.gaussian_spinor(V, seed=2007, nrhs=nrhs)
    prm = oracle.params(dims, mass=m)
    with Handle(dims, U, mass=m) as H:
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_BLOCK, lqcd.LQ_F64, nrhs=nrhs, tol=1e-10)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    for k in range(nrhs):
        assert st[k].true_rel_residual < 1e-10
        x_or, _, _, _ = oracle.cg(oracle.OP_WILSON, b[k], U, prm, 1e-12)
        assert rel_err(xg[k], x_or) < 1e-7


def test_block_cg_zero_column_is_left_out():
    """A zero right-hand side inside the block: its solution is zero and the
    other columns still converge (the block holds only unfinished columns)."""
    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    m = 0.1
    U = inputs.gauge_field(dims, "random", seed=1008)
    b = inputs.gaussian_spinor(V, seed=2008, nrhs=4)
    b[2] = 0
    with Handle(dims, U, mass=m) as H:
        bd = dev(b)
        xd = torch.full_like(bd, 7.0)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_BLOCK, lqcd.LQ_F64, nrhs=4, tol=1e-10)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0
    assert np.all(xg[2] == 0) and st[2].iters == 0
    prm = oracle.params(dims, mass=m)
    for k in (0, 1, 3):
        assert st[k].true_rel_residual < 1e-10
        assert rel_err(oracle.apply_normal(oracle.OP_WILSON, xg[k], U, prm), b[k]) < 1e-9


def test_breakdown_is_reported_and_x_is_left_intact():
    """Breakdown injected on the host: zero links and m = -4 make D = m + 4 = 0, so
    <p, A p> = |D p|^2 = 0 at the first step.  Plain FP64, mixed (FP16 inner, through
    the FP32 middle level) and mixed (FP32 inner) solves return LQ_ERR_BREAKDOWN and
    leave x as it was: zero from a zero start, the guess when one is given."""
    dims = (4, 4, 4, 4)
    U = np.zeros((256, 4, 3, 3), dtype=complex)
    b = inputs.gaussian_spinor(256, seed=2010)
    guess = inputs.gaussian_spinor(256, seed=2011)
    with Handle(dims, U, mass=-4.0) as H:
        bd = dev(b)
        for mode, inner in ((lqcd.LQ_CG_PLAIN, lqcd.LQ_F32), (lqcd.LQ_CG_MIXED, lqcd.LQ_F16),
                            (lqcd.LQ_CG_MIXED, lqcd.LQ_F32)):
            for x0 in (None, guess):
                x = torch.zeros_like(bd) if x0 is None else dev(x0)
                cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, mode, lqcd.LQ_F64, tol=1e-10, inner=inner,
                                         x0_is_guess=x0 is not None)
                rc, st = lqcd.cg_solve(H.h, x, bd, cp, check=False)
                assert rc == -6 and st[0].status == -6, (mode, inner, rc)
                want = np.zeros_like(b) if x0 is None else x0
                assert np.array_equal(host(x), want)


def test_compressed_links_must_be_su3():
    """Two-row link storage rebuilds row 3 from rows 1 and 2, which is exact only for
    SU(3): lq_create with compress12 = 1 refuses a field with a corrupted link (a
    scaled link, a link with det = -1, a NaN) with LQ_ERR_ARG and accepts SU(3) links in
    FP64 and FP32; the same corrupted field is accepted without compression."""
    import ctypes
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "random", seed=1000)
    bad = []
    u = U.copy()
    u[17, 2] *= 1.001  # |U^dag U - 1| = 2e-3
    bad.append(u)
    u = U.copy()
    u[200, 3] *= -1.0  # unitary, det = -1
    bad.append(u)
    u = U.copy()
    u[5, 0, 1, 2] = np.nan
    bad.append(u)
    L = lqcd.lib()
    for f in bad:
        prm = lqcd.make_params(dims, mass=0.1, compress12=True)
        Ud = dev(f)
        h = ctypes.c_void_p()
        assert L.lq_create(ctypes.byref(h), ctypes.byref(prm), Ud.data_ptr(), lqcd.LQ_F64, None) == -1
        assert h.value is None
        with Handle(dims, f, mass=0.1):  # no compression: no check
            pass
    for prec in (lqcd.LQ_F64, lqcd.LQ_F32):
        for kind in ("random", "smooth", "unit"):
            with Handle(dims, inputs.gauge_field(dims, kind, seed=1001), mass=0.1, compress12=True, U_prec=prec):
                pass


@pytest.mark.parametrize("inner", [lqcd.LQ_F32, lqcd.LQ_F16])
@pytest.mark.parametrize("op", ["wilson_eo", "dwf"])
def test_mixed_multi_field_solves_on_odd_tile_counts(inner, op):
    """4x6x2x8 has three 64-site tiles per parity, so the FP32 multi-field hop fills the
    last fused-norm slots of the 128-site layout with zeros: batched mixed CG of three
    even-odd sources (FP32 and FP16 inner), and the domain-wall CG (Ls = 5, FP32 inner),
    each solution checked through the oracle's operator."""
    dims = (4, 6, 2, 8)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1006)
    if op == "wilson_eo":
        m = 0.05
        b = inputs.gaussian_spinor(V // 2, seed=2020, nrhs=3)
        prm = oracle.params(dims, mass=m)
        kw, opc, ocode, n = dict(mass=m), lqcd.LQ_OP_WILSON_EO_NORMAL, oracle.OP_WILSON_EO, 3
    else:
        if inner != lqcd.LQ_F32:
            pytest.skip("the domain-wall mixed solve takes FP32 inner solves")
        Ls = 5
        prm = oracle.params(dims, Ls=Ls, M5=1.8, mf=0.01)
        b = inputs.gaussian_spinor(V, seed=2021, nrhs=Ls)
        kw, opc, ocode, n = dict(Ls=Ls, M5=1.8, mf=0.01), lqcd.LQ_OP_DWF_NORMAL, oracle.OP_DWF, 1
    with Handle(dims, U, **kw) as H:
        bd = dev(b)
        xd = torch.zeros_like(bd)
        cp = lqcd.make_cg_params(opc, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=n, tol=1e-10, inner=inner,
                                 inner_tol=1e-6 if op == "dwf" else 0.0)
        rc, st = lqcd.cg_solve(H.h, xd, bd, cp)
        xg = host(xd)
    assert rc == 0 and all(s.true_rel_residual < 1e-10 for s in st)
    if op == "wilson_eo":
        for k in range(3):
            assert rel_err(oracle.apply_normal(ocode, xg[k], U, prm), b[k]) <= 1e-10
    else:
        assert rel_err(oracle.apply_normal(ocode, xg, U, prm), b) <= 1e-10
