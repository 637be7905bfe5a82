"""The algebra behind the spin-projected halo faces (lq_face_pack /
lq_face_unpack), checked on the CPU in the oracle's own gamma basis: a hop
reads a ghost site only through (1 + S gamma_t); with h = psi_up + S psi_dn the
ghost chi = [h/2; S h/2] has the same projection as psi for both signs, and so
does the 16-bit form [h; S h] with the site norm halved; h carries half the
numbers of psi; and the projection of the other sign is not preserved (the
ghost serves only the hop direction it was packed for)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("S", [1, -1])
def test_ghost_has_the_projection_of_the_spinor(S):
    gt = oracle.gamma(3)
    rng = np.random.default_rng(7)
    psi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    proj = np.eye(4) + S * gt
    h = psi[0:2] + S * psi[2:4]
    chi = np.concatenate([h / 2, S * h / 2])
    assert np.allclose(proj @ chi, proj @ psi, rtol=0, atol=1e-14)
    # 16-bit form: stored components [h; S h], norm n/2 (the decoded spinor is the same chi)
    n = np.max(np.abs(np.concatenate([psi.real, psi.imag])))
    stored, norm = np.concatenate([h, S * h]) / n, n / 2
    assert np.allclose(proj @ (stored * norm), proj @ psi, rtol=0, atol=1e-14)
    # h is half the spinor's numbers, and the upper rows of the projection are h itself
    assert h.size * 2 == psi.size
    assert np.allclose((proj @ psi)[0:2], h, rtol=0, atol=1e-14)
    # the opposite projector sees a different spinor
    other = np.eye(4) - S * gt
    assert not np.allclose(other @ chi, other @ psi)
