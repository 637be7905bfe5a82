"""Pins that tie the CPU oracle to the mathematics, not to itself.

Each test checks the oracle against something it does not compute: a closed
form (the free-field plane-wave spectrum), an algebraic identity (Clifford
algebra, adjointness, gamma_5-hermiticity, gauge covariance, Gamma_5 R_5
hermiticity of the domain-wall operator), a special case that reduces to
another operator (domain wall at Ls = 1), or a library solver (numpy dense LU).
The mistakes each one catches are listed in its docstring.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2001_07557_gb300 import inputs

BC_T = (1, 1, 1, -1)

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
]


def chiral_gammas():
    """The basis read for the operator: gamma_k = [[0,-i s_k],[i s_k,0]], gamma_t = [[0,1],[1,0]]."""
    z = np.zeros((2, 2), dtype=complex)
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in SIGMA]
    g.append(np.block([[z, np.eye(2)], [np.eye(2), z]]))
    return g


def coords(dims):
    L0, L1, L2, L3 = dims
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1), np.arange(L0), indexing="ij")
    return np.stack([x0.ravel(), x1.ravel(), x2.ravel(), x3.ravel()], axis=1)


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# ------------------------------------------------------------------ gammas


def test_gamma_clifford_algebra(orc):
    """{gamma_mu, gamma_nu} = 2 delta, hermitian, gamma_5 = gamma_x gamma_y gamma_z gamma_t = diag(1,1,-1,-1)."""
    g = [orc.gamma(mu) for mu in range(4)]
    for mu, nu in itertools.product(range(4), range(4)):
        ac = g[mu] @ g[nu] + g[nu] @ g[mu]
        np.testing.assert_allclose(ac, 2.0 * np.eye(4) * (mu == nu), atol=1e-15)
    for mu in range(4):
        np.testing.assert_allclose(g[mu], g[mu].conj().T, atol=1e-15)
        np.testing.assert_allclose(g[mu], chiral_gammas()[mu], atol=1e-15)
    g5 = orc.gamma(4)
    np.testing.assert_allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    np.testing.assert_allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)


# ------------------------------------------------------------- free field


def plane_wave(dims, bc, n, rng):
    """e^{i p.x} u with p_mu = 2 pi (n_mu + theta_mu) / L_mu, theta = 1/2 where bc = -1."""
    p = np.array([2 * math.pi * (n[mu] + (0.5 if bc[mu] < 0 else 0.0)) / dims[mu] for mu in range(4)])
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    ph = np.exp(1j * coords(dims) @ p)
    return ph[:, None, None] * u[None], p, u, ph


@pytest.mark.parametrize("dims,bc", [((4, 6, 2, 8), BC_T), ((6, 4, 4, 2), (-1, 1, 1, 1)),
                                      ((2, 2, 2, 2), BC_T)])
@pytest.mark.parametrize("r", [1.0, 0.7])
def test_free_field_closed_form(orc, dims, bc, r):
    """Unit links: D e^{ipx}u = e^{ipx}[m + r sum(1 - cos p) + i sum gamma_mu sin p_mu] u.

    Fixes the gamma basis, the sign of the gamma term, the 1/2, r, the
    boundary phases and every neighbour offset (the momenta differ per
    direction and L0 != L1).  The dagger must give the conjugate symbol.
    """
    rng = np.random.default_rng(7)
    U = inputs.gauge_field(dims, "unit")
    m = 0.1
    G = chiral_gammas()
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (3, 1, 0, 1)]:
        n = tuple(k % d for k, d in zip(n, dims))
        psi, p, u, ph = plane_wave(dims, bc, n, rng)
        a = m + r * np.sum(1 - np.cos(p))
        S = sum(np.sin(p[mu]) * G[mu] for mu in range(4))
        for dag in (False, True):
            sym = a * np.eye(4) + (-1j if dag else 1j) * S
            want = ph[:, None, None] * (sym @ u)[None]
            got = orc.wilson_dslash(psi, U, dims, m, bc=bc, r=r, dagger=dag)
            assert rel(got, want) < 1e-14


# --------------------------------------------------- adjoint, gamma5-hermiticity


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 2)])
def test_dagger_is_adjoint_and_gamma5_hermitian(orc, dims):
    """<y, D x> = <D^dag y, x> and D^dag = gamma_5 D gamma_5 with random SU(3) links.

    Catches a wrong projector in the dagger, a missing conjugate on the
    backward link, and a hop that is not the transpose of the other.
    """
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=11)
    x = inputs.gaussian_spinor(V, seed=12)
    y = inputs.gaussian_spinor(V, seed=13)
    Dx = orc.wilson_dslash(x, U, dims, 0.1)
    Ddy = orc.wilson_dslash(y, U, dims, 0.1, dagger=True)
    assert abs(vdot(y, Dx) - vdot(Ddy, x)) / abs(vdot(y, Dx)) < 1e-13
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    g5y = np.einsum("ab,sbc->sac", g5, y)
    want = np.einsum("ab,sbc->sac", g5, orc.wilson_dslash(g5y, U, dims, 0.1))
    assert rel(Ddy, want) < 1e-14


# --------------------------------------------------------- gauge covariance


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 6, 4, 4)])
def test_gauge_covariance(orc, dims):
    """D[U^g](g psi) = g D[U] psi, U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag.

    Catches U vs U^dag or U^T, U_mu(x) vs U_mu(x-mu) on the backward hop, and
    a link read from the wrong site; the antiperiodic phase stays outside U.
    """
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=21)
    g = inputs.random_su3(V, np.random.default_rng(3000))
    psi = inputs.gaussian_spinor(V, seed=22)
    X = coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        xp = X.copy()
        xp[:, mu] = (xp[:, mu] + 1) % dims[mu]
        ip = xp[:, 0] + dims[0] * (xp[:, 1] + dims[1] * (xp[:, 2] + dims[2] * xp[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[ip], 1, 2))
    psig = np.einsum("xij,xsj->xsi", g, psi)
    for dag in (False, True):
        lhs = orc.wilson_dslash(psig, Ug, dims, 0.05, dagger=dag)
        rhs = np.einsum("xij,xsj->xsi", g, orc.wilson_dslash(psi, U, dims, 0.05, dagger=dag))
        assert rel(lhs, rhs) < 1e-14


# -------------------------------------------------------------- dense 2^4


def sorted_spectrum(ev, decimals=9):
    """Eigenvalues sorted after rounding, so that rounding noise cannot reorder them."""
    ev = np.round(np.asarray(ev), decimals)
    return ev[np.lexsort((ev.imag, ev.real))]


def dense(apply, n_sites):
    n = n_sites * 12
    M = np.empty((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for k in range(n):
        e[:] = 0
        e[k] = 1
        M[:, k] = apply(e.reshape(n_sites, 4, 3)).ravel()
    return M


def test_dense_2444_free_spectrum(orc):
    """Dense D on 2^4 with unit links: spectrum {m + r(2n+1) +- i}, multiplicity 12 C(3, n).

    On L = 2 the forward and backward neighbours are the same site, so this
    also fixes how the two hops accumulate.
    """
    dims = (2, 2, 2, 2)
    m = 0.1
    U = inputs.gauge_field(dims, "unit")
    D = dense(lambda v: orc.wilson_dslash(v, U, dims, m), 16)
    ev = np.linalg.eigvals(D)
    want = []
    for n in range(4):
        for s in (+1, -1):
            want += [m + (2 * n + 1) + 1j * s] * (12 * math.comb(3, n))
    np.testing.assert_allclose(sorted_spectrum(ev), sorted_spectrum(want), atol=1e-9)


def test_dense_2444_random_links(orc):
    """Dense D on 2^4 with random links: D^dag (conjugate transpose) = the dagger apply = g5 D g5,
    and the spectrum is closed under complex conjugation."""
    dims = (2, 2, 2, 2)
    U = inputs.gauge_field(dims, "random", seed=31)
    D = dense(lambda v: orc.wilson_dslash(v, U, dims, 0.1), 16)
    Dd = dense(lambda v: orc.wilson_dslash(v, U, dims, 0.1, dagger=True), 16)
    np.testing.assert_allclose(Dd, D.conj().T, atol=1e-14)
    G5 = np.kron(np.eye(16), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    np.testing.assert_allclose(G5 @ D @ G5, Dd, atol=1e-14)
    ev = np.linalg.eigvals(D)
    np.testing.assert_allclose(sorted_spectrum(ev), sorted_spectrum(ev.conj()), atol=1e-8)


# ------------------------------------------------------------- even-odd


def test_even_odd_schur_solve_matches_full_solve(orc):
    """Mhat x_e = b_e + 1/(2a) H_eo b_o, x_o = (b_o + 1/2 H_oe x_e)/a reproduces the
    dense LU solution of D x = b (catches a wrong Schur coefficient or sign)."""
    dims = (4, 2, 2, 4)
    V = int(np.prod(dims))
    m = 0.2
    a = m + 4
    U = inputs.gauge_field(dims, "random", seed=41)
    b = inputs.gaussian_spinor(V, seed=42)
    D = dense(lambda v: orc.wilson_dslash(v, U, dims, m), V)
    x_ref = np.linalg.solve(D, b.ravel()).reshape(V, 4, 3)
    be, bo = inputs.to_half(b, dims, 0), inputs.to_half(b, dims, 1)
    bhat = be + orc.wilson_hop_eo(bo, U, dims, 0) / (2 * a)
    M = dense(lambda v: orc.wilson_schur(v, U, dims, m), V // 2)
    xe = np.linalg.solve(M, bhat.ravel()).reshape(V // 2, 4, 3)
    xo = (bo + 0.5 * orc.wilson_hop_eo(xe, U, dims, 1)) / a
    assert rel(inputs.from_halves(xe, xo, dims), x_ref) < 1e-12
    Md = dense(lambda v: orc.wilson_schur(v, U, dims, m, dagger=True), V // 2)
    np.testing.assert_allclose(Md, M.conj().T, atol=1e-14)


def test_eo_hop_is_block_of_full_hop(orc):
    dims = (4, 4, 2, 2)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=43)
    psi = inputs.gaussian_spinor(V, seed=44)
    full = orc.wilson_hop(psi, U, dims)
    for p in (0, 1):
        src = inputs.to_half(psi, dims, 1 - p)
        emb = inputs.from_halves(src, np.zeros_like(src), dims) if p == 1 else \
            inputs.from_halves(np.zeros_like(src), src, dims)
        np.testing.assert_allclose(orc.wilson_hop_eo(src, U, dims, p),
                                   inputs.to_half(orc.wilson_hop(emb, U, dims), dims, p), atol=1e-14)
    assert full.shape == psi.shape


# ------------------------------------------------------------------- CG


def test_cg_plane_wave_one_iteration(orc):
    """(D^dag D) e^{ipx}u = (a^2 + sum sin^2 p) e^{ipx}u: CG converges in one step."""
    dims = (4, 4, 4, 8)
    rng = np.random.default_rng(5)
    U = inputs.gauge_field(dims, "unit")
    b, p, u, ph = plane_wave(dims, BC_T, (1, 0, 2, 3), rng)
    m = 0.1
    lam = (m + np.sum(1 - np.cos(p))) ** 2 + np.sum(np.sin(p) ** 2)
    prm = orc.params(dims, mass=m)
    x, it, res, rc = orc.cg(orc.OP_WILSON, b, U, prm, 1e-12)
    assert rc == orc.OK and it == 1
    assert rel(x, b / lam) < 1e-13


def test_cg_matches_dense_lu_on_4444(orc):
    """4^4 random SU(3), m = 0.1, CG on D^dag D to 1e-12 vs numpy's dense LU of D x = eta."""
    dims = (4, 4, 4, 4)
    V = 256
    U = inputs.gauge_field(dims, "random", seed=1000)
    eta = inputs.gaussian_spinor(V, seed=2000)
    D = dense(lambda v: orc.wilson_dslash(v, U, dims, 0.1), V)
    x_ref = np.linalg.solve(D, eta.ravel()).reshape(V, 4, 3)
    prm = orc.params(dims, mass=0.1)
    b = orc.wilson_dslash(eta, U, dims, 0.1, dagger=True)
    x, it, res, rc = orc.cg(orc.OP_WILSON, b, U, prm, 1e-12)
    assert rc == orc.OK and res < 1e-12
    sv = np.linalg.svd(D, compute_uv=False)
    kappa = (sv[0] / sv[-1]) ** 2
    assert rel(x, x_ref) < 1e-12 * kappa
    assert rel(orc.wilson_dslash(x, U, dims, 0.1), eta) < 1e-10


# ----------------------------------------------------------- domain wall


def test_dwf_ls1_is_wilson(orc):
    """Ls = 1: the wall terms fold into a mass, D_dw = D_W(1 - M5 + mf)."""
    dims = (4, 2, 4, 2)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=51)
    psi = inputs.gaussian_spinor(V, seed=52)
    for dag in (False, True):
        got = orc.dwf_dslash(psi[None], U, dims, 1, 1.8, 0.01, dagger=dag)[0]
        want = orc.wilson_dslash(psi, U, dims, 1 - 1.8 + 0.01, dagger=dag)
        assert rel(got, want) < 1e-14


def test_dwf_free_field_closed_form(orc):
    """Unit links, psi(x, s) = e^{ipx} u_s: the 4Ls x 4Ls symbol
    [(1 - M5 + sum(1 - cos p)) + i gamma.sin p] x 1 - P- x S+ - P+ x S-,
    (S+)_{s,s+1} = 1, (S+)_{Ls-1,0} = -mf, (S-)_{s,s-1} = 1, (S-)_{0,Ls-1} = -mf."""
    dims = (4, 4, 2, 4)
    Ls, M5, mf = 6, 1.8, 0.01
    rng = np.random.default_rng(9)
    U = inputs.gauge_field(dims, "unit")
    G = chiral_gammas()
    g5 = G[0] @ G[1] @ G[2] @ G[3]
    Pp, Pm = (np.eye(4) + g5) / 2, (np.eye(4) - g5) / 2
    Sp = np.diag(np.ones(Ls - 1), 1).astype(complex)
    Sp[Ls - 1, 0] = -mf
    Sm = Sp.T.copy()
    for n in [(0, 0, 0, 0), (1, 3, 1, 2)]:
        _, p, _, ph = plane_wave(dims, BC_T, n, rng)
        us = rng.standard_normal((Ls, 4, 3)) + 1j * rng.standard_normal((Ls, 4, 3))
        psi5 = ph[None, :, None, None] * us[:, None]
        w = (1 - M5 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(np.sin(p[m]) * G[m] for m in range(4))
        for dag in (False, True):
            if dag:
                w_ = w.conj().T
                K = np.kron(np.eye(Ls), w_) - np.kron(Sm, Pm) - np.kron(Sp, Pp)
            else:
                K = np.kron(np.eye(Ls), w) - np.kron(Sp, Pm) - np.kron(Sm, Pp)
            want_u = (K @ us.reshape(Ls * 4, 3)).reshape(Ls, 4, 3)
            want = ph[None, :, None, None] * want_u[:, None]
            got = orc.dwf_dslash(psi5, U, dims, Ls, M5, mf, dagger=dag)
            assert rel(got, want) < 1e-14


def test_dwf_gamma5_r5_hermiticity(orc):
    """D_dw^dag = Gamma5 R5 D_dw Gamma5 R5, (R5 psi)(s) = psi(Ls-1-s), and <y, D x> = <D^dag y, x>."""
    dims = (2, 4, 2, 4)
    V = int(np.prod(dims))
    Ls = 5
    U = inputs.gauge_field(dims, "random", seed=61)
    x = inputs.gaussian_spinor(V, seed=62, nrhs=Ls)
    y = inputs.gaussian_spinor(V, seed=63, nrhs=Ls)
    Dx = orc.dwf_dslash(x, U, dims, Ls, 1.8, 0.01)
    Ddy = orc.dwf_dslash(y, U, dims, Ls, 1.8, 0.01, dagger=True)
    assert abs(vdot(y, Dx) - vdot(Ddy, x)) / abs(vdot(y, Dx)) < 1e-13
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])

    def g5r5(v):
        return np.einsum("ab,svbc->svac", g5, v[::-1])

    assert rel(Ddy, g5r5(orc.dwf_dslash(np.ascontiguousarray(g5r5(y)), U, dims, Ls, 1.8, 0.01))) < 1e-14


def test_dwf_cg_small(orc):
    """CG on D_dw^dag D_dw reaches 1e-10 and the solution solves D_dw x = eta."""
    dims = (4, 4, 2, 2)
    V = int(np.prod(dims))
    Ls = 4
    U = inputs.gauge_field(dims, "smooth", seed=1004)
    eta = inputs.gaussian_spinor(V, seed=2004, nrhs=Ls)
    prm = orc.params(dims, Ls=Ls, M5=1.8, mf=0.01)
    b = orc.apply_op(orc.OP_DWF, eta, U, prm, dagger=True)
    x, it, res, rc = orc.cg(orc.OP_DWF, b, U, prm, 1e-10)
    assert rc == orc.OK
    assert rel(orc.apply_op(orc.OP_DWF, x, U, prm), eta) < 1e-8


# ------------------------------------------------- domain wall, even-odd


def dense_map(fn, n):
    """The matrix of a linear map on C^n, column by column."""
    M = np.zeros((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = fn(e).ravel()
    return M


def test_mobius_reduces_to_shamir_and_its_c5_term_is_dw_times_s(orc):
    """Moebius D_M(b5, c5): b5 = 1, c5 = 0 gives the Shamir operator (a separate
    code path); D_M is affine in (b5, c5), its b5 part is D_W on every slice and
    its c5 part is D_W applied to S psi, where S psi = -M5op(psi) at M5 = 5 comes
    from the pinned site-local operator; the dagger is the adjoint."""
    dims, Ls, M5, mf = (2, 2, 2, 4), 4, 1.8, 0.07
    V = 32
    U = inputs.gauge_field(dims, "random", seed=31)
    psi = inputs.gaussian_spinor(V, seed=32, nrhs=Ls)
    y = inputs.gaussian_spinor(V, seed=33, nrhs=Ls)
    for dag in (False, True):
        shamir = orc.dwf_dslash(psi, U, dims, Ls, M5, mf, dagger=dag)
        assert rel(orc.dwf_mobius_dslash(psi, U, dims, Ls, M5, mf, 1.0, 0.0, dagger=dag), shamir) < 1e-14
    D = lambda b5, c5: orc.dwf_mobius_dslash(psi, U, dims, Ls, M5, mf, b5, c5)  # noqa: E731
    base = D(0.0, 0.0)
    DW = np.stack([orc.wilson_dslash(psi[s], U, dims, -M5) for s in range(Ls)])
    assert rel(D(1.0, 0.0) - base, DW) < 1e-13
    S = -orc.dwf_m5(psi, Ls, 5.0, mf)
    DWS = np.stack([orc.wilson_dslash(S[s], U, dims, -M5) for s in range(Ls)])
    assert rel(D(0.0, 1.0) - base, DWS) < 1e-13
    assert rel(D(1.5, 0.5) - base, 1.5 * DW + 0.5 * DWS) < 1e-13
    lhs = np.vdot(y.ravel(), orc.dwf_mobius_dslash(psi, U, dims, Ls, M5, mf, 1.5, 0.5).ravel())
    rhs = np.vdot(orc.dwf_mobius_dslash(y, U, dims, Ls, M5, mf, 1.5, 0.5, dagger=True).ravel(), psi.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_dwf_m5_is_the_zero_link_operator(orc):
    """M5 (the site-local part of D_dw) equals D_dw with all links zero, where
    the 4-d hop vanishes; also for the dagger.  Catches a wrong diagonal
    (5 - M5), swapped projectors or a wall sign in M5."""
    dims, Ls, M5, mf = (2, 2, 2, 4), 5, 1.8, 0.07
    V = 32
    U0 = np.zeros((V, 4, 3, 3), dtype=complex)
    psi = inputs.gaussian_spinor(V, seed=21, nrhs=Ls)
    for dag in (False, True):
        want = orc.dwf_dslash(psi, U0, dims, Ls, M5, mf, dagger=dag)
        assert rel(orc.dwf_m5(psi, Ls, M5, mf, dagger=dag), want) < 1e-15
        assert rel(orc.dwf_m5_inv(orc.dwf_m5(psi, Ls, M5, mf, dag), Ls, M5, mf, dag), psi) < 1e-13


def test_dwf_eo_schur_solve_matches_full_solve(orc):
    """Solving D_dw psi = eta through the even-odd Schur complement (source
    preparation, dense solve of Mhat, reconstruction of the odd half) gives
    numpy's dense solve of the full D_dw.  Catches a sign or a missing factor
    in Mhat, in the prepared source or in the reconstruction, and a wrong M5^{-1}."""
    dims, Ls, M5, mf = (2, 2, 2, 4), 4, 1.8, 0.05
    V = 32
    U = inputs.gauge_field(dims, "random", seed=22)
    eta = inputs.gaussian_spinor(V, seed=23, nrhs=Ls)
    D = dense_map(lambda v: orc.dwf_dslash(v.reshape(Ls, V, 4, 3), U, dims, Ls, M5, mf), Ls * V * 12)
    psi = np.linalg.solve(D, eta.ravel()).reshape(Ls, V, 4, 3)
    M = dense_map(lambda v: orc.dwf_schur(v.reshape(Ls, V // 2, 4, 3), U, dims, Ls, M5, mf), Ls * V // 2 * 12)
    bhat = orc.dwf_eo_prepare(eta, U, dims, Ls, M5, mf)
    xe = np.linalg.solve(M, bhat.ravel()).reshape(Ls, V // 2, 4, 3)
    assert rel(orc.dwf_eo_reconstruct(xe, eta, U, dims, Ls, M5, mf), psi) < 1e-12
    # the dagger is the adjoint
    Md = dense_map(lambda v: orc.dwf_schur(v.reshape(Ls, V // 2, 4, 3), U, dims, Ls, M5, mf, dagger=True),
               Ls * V // 2 * 12)
    assert np.max(np.abs(Md - M.conj().T)) < 1e-13 * np.max(np.abs(M))


def test_dwf_eo_cg_small(orc):
    """CG on Mhat^dag Mhat converges and solves the system it was given."""
    dims, Ls, M5, mf = (4, 4, 2, 4), 4, 1.8, 0.1
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=24)
    b = inputs.gaussian_spinor(V // 2, seed=25, nrhs=Ls)
    prm = orc.params(dims, Ls=Ls, M5=M5, mf=mf)
    x, it, res, rc = orc.cg(orc.OP_DWF_EO, b, U, prm, 1e-10)
    assert rc == orc.OK and res < 1e-10
    assert rel(orc.apply_normal(orc.OP_DWF_EO, x, U, prm), b) < 1e-9


def test_mobius_m5_is_the_zero_link_operator(orc):
    """The Moebius site-local part M5_M equals D_M with all links zero (the 4-d
    hop vanishes), for several (b5, c5) and the dagger; its inverse inverts it.
    Catches a wrong diagonal (4 - M5) b5 + 1, a wrong shift coefficient
    (4 - M5) c5 - 1, or S in place of S^dag."""
    dims, Ls, M5, mf = (2, 2, 2, 4), 5, 1.8, 0.07
    V = 32
    U0 = np.zeros((V, 4, 3, 3), dtype=complex)
    psi = inputs.gaussian_spinor(V, seed=41, nrhs=Ls)
    for b5, c5 in [(1.0, 0.0), (1.5, 0.5), (2.0, 1.0), (0.8, -0.3)]:
        for dag in (False, True):
            want = orc.dwf_mobius_dslash(psi, U0, dims, Ls, M5, mf, b5, c5, dagger=dag)
            m5 = orc.dwf_mobius_m5(psi, Ls, M5, mf, b5, c5, dagger=dag)
            assert rel(m5, want) < 1e-15
            assert rel(orc.dwf_mobius_m5_inv(m5, Ls, M5, mf, b5, c5, dagger=dag), psi) < 1e-13


def test_mobius_eo_schur_solve_matches_full_solve(orc):
    """Solving D_M psi = eta for the Moebius operator through its even-odd Schur
    complement (prepared source, dense solve of Mhat, reconstruction of the odd
    half) gives numpy's dense solve of the full D_M, whose own pins tie it to
    D_W and the Shamir operator; the daggered Mhat is the adjoint of Mhat, and
    Mhat equals the Schur complement numpy forms from the blocks of the dense
    D_M.  Catches B applied after the hop instead of before, a missing B in
    M_eo or M_oe, a wrong M5_M, and sign errors in the three formulas."""
    dims, Ls, M5, mf, b5, c5 = (2, 2, 2, 4), 4, 1.8, 0.05, 1.5, 0.5
    V = 32
    n = Ls * V * 12
    U = inputs.gauge_field(dims, "random", seed=42)
    eta = inputs.gaussian_spinor(V, seed=43, nrhs=Ls)
    D = dense_map(lambda v: orc.dwf_mobius_dslash(v.reshape(Ls, V, 4, 3), U, dims, Ls, M5, mf, b5, c5), n)
    psi = np.linalg.solve(D, eta.ravel()).reshape(Ls, V, 4, 3)
    M = dense_map(lambda v: orc.dwf_mobius_schur(v.reshape(Ls, V // 2, 4, 3), U, dims, Ls, M5, mf, b5, c5), n // 2)
    bhat = orc.dwf_mobius_eo_prepare(eta, U, dims, Ls, M5, mf, b5, c5)
    xe = np.linalg.solve(M, bhat.ravel()).reshape(Ls, V // 2, 4, 3)
    assert rel(orc.dwf_mobius_eo_reconstruct(xe, eta, U, dims, Ls, M5, mf, b5, c5), psi) < 1e-12
    # the Schur complement of the dense operator's parity blocks
    x = coords(dims)
    par = (x.sum(axis=1) % 2).astype(int)
    idx = np.arange(n).reshape(Ls, V, 12)
    ev = idx[:, par == 0, :].ravel()
    od = idx[:, par == 1, :].ravel()
    schur = D[np.ix_(ev, ev)] - D[np.ix_(ev, od)] @ np.linalg.solve(D[np.ix_(od, od)], D[np.ix_(od, ev)])
    assert np.max(np.abs(M - schur)) < 1e-12 * np.max(np.abs(schur))
    Md = dense_map(lambda v: orc.dwf_mobius_schur(v.reshape(Ls, V // 2, 4, 3), U, dims, Ls, M5, mf, b5, c5,
                                                  dagger=True), n // 2)
    assert np.max(np.abs(Md - M.conj().T)) < 1e-13 * np.max(np.abs(M))
    # b5 = 1, c5 = 0 is the Shamir Schur complement (a separate code path)
    pe = inputs.gaussian_spinor(V // 2, seed=44, nrhs=Ls)
    for dag in (False, True):
        assert rel(orc.dwf_mobius_schur(pe, U, dims, Ls, M5, mf, 1.0, 0.0, dagger=dag),
                   orc.dwf_schur(pe, U, dims, Ls, M5, mf, dagger=dag)) < 1e-14


# ------------------------------------------------------------ SU(3) x SU(3)


def test_su3_mul_matches_numpy_and_group_closure(orc):
    """The lattice-wide product C(x) = A(x) B(x) against numpy's matmul (an
    independent library routine) on general complex matrices, the identity on
    either side, (AB)^dag = B^dag A^dag, and closure of SU(3): a product of
    special unitary matrices is special unitary.  Catches transposed or
    conjugated operands, a swapped product order and dropped terms."""
    rng = np.random.default_rng(11)
    n = 37
    A = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    B = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    C = orc.su3_mul(A, B)
    assert np.max(np.abs(C - A @ B)) < 1e-13 * np.max(np.abs(C))
    eye = np.broadcast_to(np.eye(3), (n, 3, 3))
    assert np.array_equal(orc.su3_mul(A, eye), A) and np.array_equal(orc.su3_mul(eye, B), B)
    dag = lambda M: np.conj(np.swapaxes(M, 1, 2))  # noqa: E731
    assert np.max(np.abs(dag(C) - orc.su3_mul(dag(B), dag(A)))) < 1e-13 * np.max(np.abs(C))
    U = inputs.gauge_field((2, 2, 2, 2), "random", seed=7).reshape(-1, 3, 3)
    W = inputs.gauge_field((2, 2, 2, 2), "smooth", seed=8).reshape(-1, 3, 3)
    P = orc.su3_mul(U, W)
    assert np.max(np.abs(dag(P) @ P - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(P) - 1)) < 1e-13
    assert orc.su3_mul(np.zeros((0, 3, 3)), np.zeros((0, 3, 3))).shape == (0, 3, 3)


# ------------------------------------------------------------- generators


@pytest.mark.parametrize("kind", ["random", "smooth"])
def test_su3_generators(kind):
    U = inputs.gauge_field((2, 2, 2, 4), kind, seed=5).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.max(np.abs(np.conj(np.swapaxes(U, 1, 2)) @ U - eye)) < 1e-13
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-13
    if kind == "smooth":
        d = np.linalg.norm(U - eye, axis=(1, 2))
        assert 0.05 < d.mean() < 1.0


def test_point_sources():
    b = inputs.point_sources(16)
    assert b.shape == (12, 16, 4, 3)
    assert np.all(b.reshape(12, -1).sum(axis=1) == 1)
    assert b[5, 0, 1, 2] == 1
