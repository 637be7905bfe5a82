"""FP64 CPU oracle for the Wilson / domain-wall Dirac operators and CG.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg call this package; the library product never does.  It wraps
``wilson_oracle.c`` (plain C99 complex arithmetic, dense gamma matrices, OpenMP
over sites) through ctypes.  The conventions it follows are listed at the top
of that file; the pins that tie it to the mathematics live in
``tests/test_oracle_pins.py``.

Arrays are numpy complex128, C-contiguous, in the site-major layouts:
spinor [V][4][3], half spinor [V/2][4][3] (cb = lexi/2), gauge [V][4][3][3],
5-d spinor [Ls][V][4][3], a field of colour matrices [n][3][3].
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OP_WILSON = 0
OP_WILSON_EO = 1
OP_DWF = 2
OP_DWF_EO = 3

OK = 0
NOT_CONVERGED = -3


class Params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int * 4),
        ("bc", ctypes.c_int * 4),
        ("mass", ctypes.c_double),
        ("r", ctypes.c_double),
        ("Ls", ctypes.c_int),
        ("M5", ctypes.c_double),
        ("mf", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, OpenMP); returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _configure(L):
    p = ctypes.c_void_p
    i4 = ctypes.POINTER(ctypes.c_int)
    d = ctypes.c_double
    i = ctypes.c_int
    L.orc_gamma.argtypes = [i, p]
    L.orc_wilson_hop.argtypes = [p, p, p, i4, i4, d, i]
    L.orc_wilson_dslash.argtypes = [p, p, p, i4, i4, d, d, i]
    L.orc_wilson_hop_eo.argtypes = [p, p, p, i4, i4, d, i, i]
    L.orc_wilson_hop_eo.restype = i
    L.orc_wilson_schur.argtypes = [p, p, p, i4, i4, d, d, i]
    L.orc_wilson_schur.restype = i
    L.orc_dwf_dslash.argtypes = [p, p, p, i4, i4, i, d, d, i]
    L.orc_dwf_dslash.restype = i
    L.orc_apply_op.argtypes = [i, p, p, p, ctypes.POINTER(Params), i]
    L.orc_apply_op.restype = i
    L.orc_apply_normal.argtypes = [i, p, p, p, ctypes.POINTER(Params)]
    L.orc_apply_normal.restype = i
    L.orc_cg.argtypes = [i, p, p, p, ctypes.POINTER(Params), d, i, i4, ctypes.POINTER(d)]
    L.orc_cg.restype = i
    L.orc_su3_mul.argtypes = [p, p, p, ctypes.c_long]
    L.orc_dwf_mobius_dslash.argtypes = [p, p, p, i4, i4, i, d, d, d, d, i]
    L.orc_dwf_mobius_dslash.restype = i
    L.orc_dwf_m5.argtypes = [p, p, ctypes.c_long, i, d, d, i]
    L.orc_dwf_m5_inv.argtypes = [p, p, ctypes.c_long, i, d, d, i]
    L.orc_dwf_m5_inv.restype = i
    L.orc_dwf_schur.argtypes = [p, p, p, i4, i4, i, d, d, i]
    L.orc_dwf_schur.restype = i
    L.orc_dwf_eo_prepare.argtypes = [p, p, p, i4, i4, i, d, d]
    L.orc_dwf_eo_prepare.restype = i
    L.orc_dwf_eo_reconstruct.argtypes = [p, p, p, p, i4, i4, i, d, d]
    L.orc_dwf_eo_reconstruct.restype = i
    L.orc_dwf_mobius_m5.argtypes = [p, p, ctypes.c_long, i, d, d, d, d, i]
    L.orc_dwf_mobius_m5_inv.argtypes = [p, p, ctypes.c_long, i, d, d, d, d, i]
    L.orc_dwf_mobius_m5_inv.restype = i
    L.orc_dwf_mobius_schur.argtypes = [p, p, p, i4, i4, i, d, d, d, d, i]
    L.orc_dwf_mobius_schur.restype = i
    L.orc_dwf_mobius_eo_prepare.argtypes = [p, p, p, i4, i4, i, d, d, d, d]
    L.orc_dwf_mobius_eo_prepare.restype = i
    L.orc_dwf_mobius_eo_reconstruct.argtypes = [p, p, p, p, i4, i4, i, d, d, d, d]
    L.orc_dwf_mobius_eo_reconstruct.restype = i
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


@contextlib.contextmanager
def swapped_library(path):
    """Run the wrappers below against another build of the oracle source
    (used by the tests that plant a mistake in a copy and expect a pin to fail)."""
    global _lib
    saved = lib()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i4(v):
    return (ctypes.c_int * 4)(*[int(t) for t in v])


def _vol(dims):
    return int(np.prod(dims))


def gamma(mu: int) -> np.ndarray:
    """gamma_mu for mu = 0..3 (x, y, z, t); mu = 4 gives gamma_5."""
    g = np.zeros((4, 4), dtype=np.complex128)
    lib().orc_gamma(mu, _ptr(g))
    return g


def wilson_hop(psi, U, dims, bc=(1, 1, 1, -1), r=1.0, dagger=False):
    psi, U = _c(psi), _c(U)
    out = np.empty_like(psi)
    lib().orc_wilson_hop(_ptr(out), _ptr(psi), _ptr(U), _i4(dims), _i4(bc), r, int(dagger))
    return out


def wilson_dslash(psi, U, dims, mass, bc=(1, 1, 1, -1), r=1.0, dagger=False):
    """D psi on full fields; psi may carry leading RHS axes."""
    psi, U = _c(psi), _c(U)
    V = _vol(dims)
    flat = psi.reshape(-1, V, 4, 3)
    out = np.empty_like(flat)
    for k in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[k])
        dst = np.empty_like(src)
        lib().orc_wilson_dslash(_ptr(dst), _ptr(src), _ptr(U), _i4(dims), _i4(bc), mass, r, int(dagger))
        out[k] = dst
    return out.reshape(psi.shape)


def wilson_hop_eo(psi_half, U, dims, out_parity, bc=(1, 1, 1, -1), r=1.0, dagger=False):
    """H_{p,1-p} on half fields: output sites of parity out_parity."""
    psi_half, U = _c(psi_half), _c(U)
    V = _vol(dims)
    flat = psi_half.reshape(-1, V // 2, 4, 3)
    out = np.empty_like(flat)
    for k in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[k])
        dst = np.empty_like(src)
        rc = lib().orc_wilson_hop_eo(_ptr(dst), _ptr(src), _ptr(U), _i4(dims), _i4(bc), r, int(dagger),
                                     int(out_parity))
        assert rc == OK, rc
        out[k] = dst
    return out.reshape(psi_half.shape)


def wilson_schur(psi_e, U, dims, mass, bc=(1, 1, 1, -1), r=1.0, dagger=False):
    """Mhat psi_e = a psi_e - 1/(4a) H_eo H_oe psi_e on even half fields."""
    psi_e, U = _c(psi_e), _c(U)
    V = _vol(dims)
    flat = psi_e.reshape(-1, V // 2, 4, 3)
    out = np.empty_like(flat)
    for k in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[k])
        dst = np.empty_like(src)
        rc = lib().orc_wilson_schur(_ptr(dst), _ptr(src), _ptr(U), _i4(dims), _i4(bc), mass, r, int(dagger))
        assert rc == OK, rc
        out[k] = dst
    return out.reshape(psi_e.shape)


def dwf_dslash(psi5, U, dims, Ls, M5, mf, bc=(1, 1, 1, -1), dagger=False):
    """D_dw psi on a 5-d field [Ls][V][4][3]."""
    psi5, U = _c(psi5), _c(U)
    out = np.empty_like(psi5)
    rc = lib().orc_dwf_dslash(_ptr(out), _ptr(psi5), _ptr(U), _i4(dims), _i4(bc), int(Ls), M5, mf,
                              int(dagger))
    assert rc == OK, rc
    return out


def dwf_mobius_dslash(psi5, U, dims, Ls, M5, mf, b5, c5, bc=(1, 1, 1, -1), dagger=False):
    """Moebius D_M psi = (b5 D_W + 1) psi + (c5 D_W - 1) S psi (dagger: its adjoint) on [Ls][V][4][3]."""
    psi5, U = _c(psi5), _c(U)
    out = np.empty_like(psi5)
    rc = lib().orc_dwf_mobius_dslash(_ptr(out), _ptr(psi5), _ptr(U), _i4(dims), _i4(bc), int(Ls), M5, mf, b5, c5,
                                     int(dagger))
    assert rc == OK, rc
    return out


def dwf_m5(psi5, Ls, M5, mf, dagger=False):
    """The 4-d-site-local part of D_dw: (5 - M5) psi(s) - P- psi(s+1) - P+ psi(s-1)
    (walls -> +mf), on a 5-d field [Ls][n][4][3] of any site subset."""
    psi5 = _c(psi5)
    out = np.empty_like(psi5)
    lib().orc_dwf_m5(_ptr(out), _ptr(psi5), int(psi5.size // (12 * Ls)), int(Ls), M5, mf, int(dagger))
    return out


def dwf_m5_inv(psi5, Ls, M5, mf, dagger=False):
    """(M5)^{-1} psi (dagger: (M5^dag)^{-1}) by dense Gaussian elimination."""
    psi5 = _c(psi5)
    out = np.empty_like(psi5)
    rc = lib().orc_dwf_m5_inv(_ptr(out), _ptr(psi5), int(psi5.size // (12 * Ls)), int(Ls), M5, mf, int(dagger))
    assert rc == OK, rc
    return out


def dwf_schur(psi5e, U, dims, Ls, M5, mf, bc=(1, 1, 1, -1), dagger=False):
    """Mhat = M5 - M_eo M5^{-1} M_oe (dagger: its adjoint) on an even 5-d half field [Ls][V/2][4][3]."""
    psi5e, U = _c(psi5e), _c(U)
    out = np.empty_like(psi5e)
    rc = lib().orc_dwf_schur(_ptr(out), _ptr(psi5e), _ptr(U), _i4(dims), _i4(bc), int(Ls), M5, mf, int(dagger))
    assert rc == OK, rc
    return out


def dwf_eo_prepare(eta5, U, dims, Ls, M5, mf, bc=(1, 1, 1, -1)):
    """eta_hat_e = eta_e - M_eo M5^{-1} eta_o for a full 5-d source [Ls][V][4][3]."""
    eta5, U = _c(eta5), _c(U)
    out = np.empty((Ls, _vol(dims) // 2, 4, 3), dtype=np.complex128)
    rc = lib().orc_dwf_eo_prepare(_ptr(out), _ptr(eta5), _ptr(U), _i4(dims), _i4(bc), int(Ls), M5, mf)
    assert rc == OK, rc
    return out


def dwf_eo_reconstruct(x5e, eta5, U, dims, Ls, M5, mf, bc=(1, 1, 1, -1)):
    """The full 5-d solution: psi_e = x_e, psi_o = M5^{-1} (eta_o - M_oe x_e)."""
    x5e, eta5, U = _c(x5e), _c(eta5), _c(U)
    out = np.empty_like(eta5)
    rc = lib().orc_dwf_eo_reconstruct(_ptr(out), _ptr(x5e), _ptr(eta5), _ptr(U), _i4(dims), _i4(bc), int(Ls),
                                      M5, mf)
    assert rc == OK, rc
    return out


def dwf_mobius_m5(psi5, Ls, M5, mf, b5, c5, dagger=False):
    """The 4-d-site-local part of the Moebius operator, (4 - M5)(b5 + c5 S) + 1 - S
    (dagger: S -> S^dag), on a 5-d field [Ls][n][4][3] of any site subset."""
    psi5 = _c(psi5)
    out = np.empty_like(psi5)
    lib().orc_dwf_mobius_m5(_ptr(out), _ptr(psi5), int(psi5.size // (12 * Ls)), int(Ls), M5, mf, b5, c5,
                            int(dagger))
    return out


def dwf_mobius_m5_inv(psi5, Ls, M5, mf, b5, c5, dagger=False):
    """The inverse of dwf_mobius_m5 (dagger: of its adjoint) by dense Gaussian elimination."""
    psi5 = _c(psi5)
    out = np.empty_like(psi5)
    rc = lib().orc_dwf_mobius_m5_inv(_ptr(out), _ptr(psi5), int(psi5.size // (12 * Ls)), int(Ls), M5, mf, b5, c5,
                                     int(dagger))
    assert rc == OK, rc
    return out


def dwf_mobius_schur(psi5e, U, dims, Ls, M5, mf, b5, c5, bc=(1, 1, 1, -1), dagger=False):
    """Moebius Mhat = M5_M - M_eo M5_M^{-1} M_oe, M_eo = -1/2 H_eo (b5 + c5 S) (dagger: its
    adjoint) on an even 5-d half field [Ls][V/2][4][3]."""
    psi5e, U = _c(psi5e), _c(U)
    out = np.empty_like(psi5e)
    rc = lib().orc_dwf_mobius_schur(_ptr(out), _ptr(psi5e), _ptr(U), _i4(dims), _i4(bc), int(Ls), M5, mf, b5, c5,
                                    int(dagger))
    assert rc == OK, rc
    return out


def dwf_mobius_eo_prepare(eta5, U, dims, Ls, M5, mf, b5, c5, bc=(1, 1, 1, -1)):
    """Moebius eta_hat_e = eta_e - M_eo M5_M^{-1} eta_o for a full 5-d source [Ls][V][4][3]."""
    eta5, U = _c(eta5), _c(U)
    out = np.empty((Ls, _vol(dims) // 2, 4, 3), dtype=np.complex128)
    rc = lib().orc_dwf_mobius_eo_prepare(_ptr(out), _ptr(eta5), _ptr(U), _i4(dims), _i4(bc), int(Ls), M5, mf, b5,
                                         c5)
    assert rc == OK, rc
    return out


def dwf_mobius_eo_reconstruct(x5e, eta5, U, dims, Ls, M5, mf, b5, c5, bc=(1, 1, 1, -1)):
    """The full Moebius 5-d solution: psi_e = x_e, psi_o = M5_M^{-1} (eta_o - M_oe x_e)."""
    x5e, eta5, U = _c(x5e), _c(eta5), _c(U)
    out = np.empty_like(eta5)
    rc = lib().orc_dwf_mobius_eo_reconstruct(_ptr(out), _ptr(x5e), _ptr(eta5), _ptr(U), _i4(dims), _i4(bc),
                                             int(Ls), M5, mf, b5, c5)
    assert rc == OK, rc
    return out


def params(dims, bc=(1, 1, 1, -1), mass=0.0, r=1.0, Ls=0, M5=0.0, mf=0.0) -> Params:
    p = Params()
    p.dims = (ctypes.c_int * 4)(*[int(t) for t in dims])
    p.bc = (ctypes.c_int * 4)(*[int(t) for t in bc])
    p.mass, p.r, p.Ls, p.M5, p.mf = float(mass), float(r), int(Ls), float(M5), float(mf)
    return p


def apply_op(op, psi, U, prm: Params, dagger=False):
    """K psi for K = D (OP_WILSON), Mhat (OP_WILSON_EO) or D_dw (OP_DWF)."""
    psi, U = _c(psi), _c(U)
    out = np.empty_like(psi)
    rc = lib().orc_apply_op(op, _ptr(out), _ptr(psi), _ptr(U), ctypes.byref(prm), int(dagger))
    assert rc == OK, rc
    return out


def apply_normal(op, psi, U, prm: Params):
    """K^dag K psi."""
    psi, U = _c(psi), _c(U)
    out = np.empty_like(psi)
    rc = lib().orc_apply_normal(op, _ptr(out), _ptr(psi), _ptr(U), ctypes.byref(prm))
    assert rc == OK, rc
    return out


def cg(op, b, U, prm: Params, tol, maxiter=100000):
    """CG on K^dag K x = b from x = 0; returns (x, iterations, |r|/|b|, status)."""
    b, U = _c(b), _c(U)
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = lib().orc_cg(op, _ptr(x), _ptr(b), _ptr(U), ctypes.byref(prm), float(tol), int(maxiter),
                      ctypes.byref(it), ctypes.byref(res))
    return x, it.value, res.value, rc


def su3_mul(A, B):
    """C[x] = A[x] B[x] for fields of 3x3 complex matrices, shape (n, 3, 3):
    the lattice-wide product of the paper's SU(3) benchmark (Sec. 3.3, Fig. 4a-c)."""
    A, B = _c(A), _c(B)
    if A.shape != B.shape or A.shape[-2:] != (3, 3):
        raise ValueError("su3_mul takes two (n, 3, 3) arrays of the same shape")
    C = np.empty_like(A)
    lib().orc_su3_mul(_ptr(C), _ptr(A), _ptr(B), int(A.size // 9))
    return C
