"""Seeded synthetic inputs for the Wilson / domain-wall Dirac workloads.

This module only draws random numbers and shapes them into gauge links and
spinor fields in the library's site-major layout. It holds none of the Dirac
operator's arithmetic, so the CUDA path and the CPU oracle can both be fed
from it without sharing any of the method.

Layouts (site-major, complex numbers as interleaved (re, im) pairs):
  lexi(x) = x0 + L0*(x1 + L1*(x2 + L2*x3)), x0 fastest;
  gauge   [site][mu 4][row 3][col 3]        (U_mu(x) is the link x -> x+mu)
  spinor  [site][spin 4][colour 3]
  half    [cb][spin 4][colour 3], cb = lexi/2 over the sites of one parity
  5-d     [s][site][spin 4][colour 3]

Workload recipes (all numbers drawn with numpy's PCG64 from a stated seed):
  random SU(3): QR of a complex Gaussian 3x3 matrix (re, im ~ N(0, 1/2)),
      the phases of R's diagonal moved into Q (Haar measure, Mezzadri 2007),
      then Q divided by the principal cube root of det Q so that det = 1;
  smooth SU(3): U = exp(i*eps*H) with H = (A + A^dag)/2 minus its trace/3,
      A_ij = (N(0,1) + i N(0,1))/sqrt(2), evaluated through eigh(H);
  Gaussian spinor: every real and imaginary part ~ N(0, 1);
  point sources: one unit entry per (spin, colour) at the origin.
"""
from __future__ import annotations

import numpy as np

CHUNK = 1 << 18  # matrices per batch, bounds the temporaries of qr / eigh


def volume(dims) -> int:
    L0, L1, L2, L3 = (int(d) for d in dims)
    return L0 * L1 * L2 * L3


def _complex_gaussian(rng, shape, scale):
    z = np.empty(shape, dtype=np.complex128)
    z.real = rng.standard_normal(shape) * scale
    z.imag = rng.standard_normal(shape) * scale
    return z


def random_su3(n: int, rng) -> np.ndarray:
    """n Haar-random SU(3) matrices, shape (n, 3, 3), complex128."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        z = _complex_gaussian(rng, (e - s, 3, 3), np.sqrt(0.5))
        q, r = np.linalg.qr(z)
        d = np.diagonal(r, axis1=1, axis2=2)
        q = q * (d / np.abs(d))[:, None, :]
        det = np.linalg.det(q)
        q = q / (det ** (1.0 / 3.0))[:, None, None]
        out[s:e] = q
    return out


def smooth_su3(n: int, rng, eps: float = 0.3) -> np.ndarray:
    """n matrices exp(i*eps*H), H Gaussian traceless Hermitian; shape (n, 3, 3)."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    eye = np.eye(3)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        a = _complex_gaussian(rng, (e - s, 3, 3), np.sqrt(0.5))
        h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
        tr = np.trace(h, axis1=1, axis2=2).real / 3.0
        h = h - tr[:, None, None] * eye
        lam, v = np.linalg.eigh(h)
        ph = np.exp(1j * eps * lam)
        out[s:e] = np.einsum("nij,nj,nkj->nik", v, ph, np.conj(v))
    return out


def gauge_field(dims, kind: str = "random", seed: int = 1000, eps: float = 0.3) -> np.ndarray:
    """Gauge field in [site][mu][row][col] order, shape (V, 4, 3, 3), complex128.

    kind: "random" (Haar SU(3)), "smooth" (exp(i*eps*H)) or "unit" (U = 1).
    """
    V = volume(dims)
    if kind == "unit":
        u = np.zeros((V, 4, 3, 3), dtype=np.complex128)
        u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
        return u
    rng = np.random.default_rng(seed)
    if kind == "random":
        m = random_su3(V * 4, rng)
    elif kind == "smooth":
        m = smooth_su3(V * 4, rng, eps)
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return m.reshape(V, 4, 3, 3)


def gaussian_spinor(nsites: int, seed: int = 2000, nrhs: int | None = None) -> np.ndarray:
    """Gaussian spinor field, shape (nsites, 4, 3) or (nrhs, nsites, 4, 3)."""
    rng = np.random.default_rng(seed)
    shape = (nsites, 4, 3) if nrhs is None else (nrhs, nsites, 4, 3)
    return _complex_gaussian(rng, shape, 1.0)


def point_sources(nsites: int, site: int = 0) -> np.ndarray:
    """The 12 point sources b_{s,c}(x) = delta(x, site) delta(spin, s) delta(colour, c).

    Shape (12, nsites, 4, 3); right-hand side k = 3*s + c.
    """
    b = np.zeros((12, nsites, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            b[3 * s + c, site, s, c] = 1.0
    return b


def site_parity(dims) -> np.ndarray:
    """Parity (x0+x1+x2+x3) mod 2 of every site, in lexicographic order."""
    L0, L1, L2, L3 = (int(d) for d in dims)
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1),
                                 np.arange(L0), indexing="ij")
    return ((x0 + x1 + x2 + x3) % 2).reshape(-1)


def to_half(full: np.ndarray, dims, parity: int) -> np.ndarray:
    """Pick the sites of one parity out of a full field (site axis -3), cb = lexi/2."""
    par = site_parity(dims)
    idx = np.nonzero(par == parity)[0]
    return full[..., idx, :, :]


def from_halves(even: np.ndarray, odd: np.ndarray, dims) -> np.ndarray:
    """Inverse of to_half: interleave the two parities back into lexicographic order."""
    par = site_parity(dims)
    shape = even.shape[:-3] + (par.size,) + even.shape[-2:]
    out = np.empty(shape, dtype=even.dtype)
    out[..., np.nonzero(par == 0)[0], :, :] = even
    out[..., np.nonzero(par == 1)[0], :, :] = odd
    return out
