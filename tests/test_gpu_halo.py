"""Time-slab domain decomposition on one GPU: R ranks, each a lattice of its
own (its slab of time slices plus one ghost slice on each side), ghosts filled
from the neighbours' edge slices by lq_face_copy (with the antiperiodic sign
where the copy crosses the global time boundary), the hop on the slab's own
slices by dslash_apply_slices.  The assembled result must equal the
single-domain hop bit for bit (every site sees the same inputs in the same
order) and the oracle within the hop tolerance."""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, native_buffer, rel_err
from paper_2001_07557_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQ_F64: 1e-12, lqcd.LQ_F32: 2e-6, lqcd.LQ_F16: 2e-3}
DT = {lqcd.LQ_F64: lqcd.LQ_F64, lqcd.LQ_F32: lqcd.LQ_F32, lqcd.LQ_F16: lqcd.LQ_F32}  # site-major format of the fields


class Slabs:
    """R ranks of Lt = L3 / R time slices each, ghosts at local t = 0 and Lt + 1."""

    def __init__(self, dims, R, U, mass, bc, prec):
        L0, L1, L2, L3 = dims
        assert L3 % R == 0 and (L3 // R) % 2 == 0
        self.dims, self.R, self.Lt, self.V3 = dims, R, L3 // R, L0 * L1 * L2
        self.prec, self.nat, self.bc = prec, lqcd.LQ_NATIVE | prec, bc
        self.ldims = (L0, L1, L2, self.Lt + 2)
        Ug = U.reshape(L3, self.V3, 4, 3, 3)
        self.H = []
        for r in range(R):
            ts = [(r * self.Lt + tp - 1) % L3 for tp in range(self.Lt + 2)]
            self.H.append(Handle(self.ldims, np.ascontiguousarray(Ug[ts]).reshape(-1, 4, 3, 3), mass=mass,
                                 bc=(bc[0], bc[1], bc[2], 1)))

    def scatter(self, psi):
        """global site-major field -> native fields of the ranks (ghosts zero)"""
        pg = psi.reshape(self.dims[3], self.V3, 4, 3)
        out = []
        for r, H in enumerate(self.H):
            loc = np.zeros((self.Lt + 2, self.V3, 4, 3), dtype=complex)
            loc[1:self.Lt + 1] = pg[r * self.Lt:(r + 1) * self.Lt]
            n = native_buffer(H.h, self.prec)
            lqcd.lq_convert(H.h, n, self.nat, dev(loc.reshape(-1, 4, 3), DT[self.prec]), DT[self.prec])
            out.append(n)
        return out

    def gather(self, fields):
        """the ranks' own slices of native fields -> one global site-major field"""
        parts = []
        for H, f in zip(self.H, fields):
            y = torch.empty((self.ldims[3] * self.V3, 4, 3),
                            dtype=torch.complex128 if self.prec == lqcd.LQ_F64 else torch.complex64, device="cuda")
            lqcd.lq_convert(H.h, y, DT[self.prec], f, self.nat)
            parts.append(host(y).reshape(self.Lt + 2, self.V3, 4, 3)[1:self.Lt + 1])
        return np.concatenate(parts).reshape(-1, 4, 3)

    def exchange(self, fields, stream=None, projected=False, dagger=False):
        R, Lt = self.R, self.Lt
        if projected:
            return self.exchange_projected(fields, stream, dagger)
        for r in range(R):
            lo, hi = (r - 1) % R, (r + 1) % R
            s_lo = self.bc[3] if r == 0 else 1.0  # the copy crosses t = L3-1 -> 0
            s_hi = self.bc[3] if r == R - 1 else 1.0
            lqcd.lq_face_copy(self.H[r].h, fields[r], 0, self.H[lo].h, fields[lo], Lt, self.nat, s_lo, stream)
            lqcd.lq_face_copy(self.H[r].h, fields[r], Lt + 1, self.H[hi].h, fields[hi], 1, self.nat, s_hi, stream)

    def exchange_projected(self, fields, stream, dagger):
        """Each rank packs the projected halves of its two edge slices into send
        buffers, a copy moves each to the neighbour's receive buffer (the message
        of a real exchange), and the neighbour unpacks it into its ghost."""
        R, Lt = self.R, self.Lt
        nb = lqcd.lq_face_wire_bytes(self.H[0].h, self.nat)
        s_dn = -1 if dagger else 1  # projector of the hop that reads the ghost below the slab
        s_up = -s_dn
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            send = [[torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in range(R)]
            recv = [[torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in range(R)]
            for r in range(R):
                sc_top = self.bc[3] if r == R - 1 else 1.0  # the top slice of the last rank crosses t = L3-1 -> 0
                sc_bot = self.bc[3] if r == 0 else 1.0
                lqcd.lq_face_pack(self.H[r].h, send[r][0], fields[r], Lt, self.nat, s_dn, sc_top, stream)
                lqcd.lq_face_pack(self.H[r].h, send[r][1], fields[r], 1, self.nat, s_up, sc_bot, stream)
            for r in range(R):
                recv[r][0].copy_(send[(r - 1) % R][0], non_blocking=True)
                recv[r][1].copy_(send[(r + 1) % R][1], non_blocking=True)
            for r in range(R):
                lqcd.lq_face_unpack(self.H[r].h, fields[r], 0, recv[r][0], self.nat, s_dn, stream)
                lqcd.lq_face_unpack(self.H[r].h, fields[r], Lt + 1, recv[r][1], self.nat, s_up, stream)
            self._keep = (send, recv)  # alive until the stream has used them

    def hop(self, ins, outs, overlap=False, dagger=False, projected=False):
        if not overlap:
            self.exchange(ins, projected=projected, dagger=dagger)
            for H, i, o in zip(self.H, ins, outs):
                lqcd.dslash_apply_slices(H.h, o, i, self.nat, 1, self.Lt + 1, dagger)
            return
        # interior slices on one stream while the faces move on another, then the two edge slices
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        for H, i, o in zip(self.H, ins, outs):
            if self.Lt > 2:
                lqcd.dslash_apply_slices(H.h, o, i, self.nat, 2, self.Lt, dagger, sa)
        self.exchange(ins, sb, projected=projected, dagger=dagger)
        for H, i, o in zip(self.H, ins, outs):
            lqcd.dslash_apply_slices(H.h, o, i, self.nat, 1, 2, dagger, sb)
            lqcd.dslash_apply_slices(H.h, o, i, self.nat, self.Lt, self.Lt + 1, dagger, sb)
        torch.cuda.synchronize()

    def close(self):
        for H in self.H:
            H.close()


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16])
@pytest.mark.parametrize("R,dims", [(2, (4, 4, 4, 8)), (4, (4, 6, 2, 16)), (2, (6, 4, 4, 4))])
@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("projected", [False, True])
def test_slabs_reproduce_the_single_domain_hop(prec, R, dims, overlap, projected):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=1201)
    psi = inputs.gaussian_spinor(V, seed=2201)
    bc = (1, 1, 1, -1)
    mass = 0.1
    S = Slabs(dims, R, U, mass, bc, prec)
    try:
        ins = S.scatter(psi)
        outs = [native_buffer(H.h, prec).zero_() for H in S.H]  # ghost slices of the output are never written
        for dag in (False, True):
            S.hop(ins, outs, overlap=overlap, dagger=dag, projected=projected)
            got = S.gather(outs)
            with Handle(dims, U, mass=mass, bc=bc) as G:
                nat = lqcd.LQ_NATIVE | prec
                x = dev(psi, DT[prec])
                xn, yn = native_buffer(G.h, prec), native_buffer(G.h, prec)
                lqcd.lq_convert(G.h, xn, nat, x, DT[prec])
                (lqcd.dslash_dag_apply if dag else lqcd.dslash_apply)(G.h, yn, xn, nat, lqcd.LQ_FULL)
                y = torch.empty_like(x)
                lqcd.lq_convert(G.h, y, DT[prec], yn, nat)
                single = host(y)
            assert np.array_equal(got, single)
            assert rel_err(got, oracle.wilson_dslash(psi, U, dims, mass, bc=bc, dagger=dag)) < TOL[prec]
    finally:
        S.close()


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16])
def test_face_copy_odd_offset_swaps_parities_and_scales(prec):
    """A slice copied to a slice an odd distance away (parities of its sites
    swap between the two positions), times -1, into another field."""
    dims = (4, 2, 6, 6)
    V3 = 4 * 2 * 6
    V = V3 * 6
    U = inputs.gauge_field(dims, "unit")
    a = inputs.gaussian_spinor(V, seed=2202)
    with Handle(dims, U) as H:
        nat = lqcd.LQ_NATIVE | prec
        an, bn = native_buffer(H.h, prec), native_buffer(H.h, prec)
        lqcd.lq_convert(H.h, an, nat, dev(a, DT[prec]), DT[prec])
        lqcd.lq_convert(H.h, bn, nat, dev(np.zeros_like(a), DT[prec]), DT[prec])
        lqcd.lq_face_copy(H.h, bn, 4, H.h, an, 1, nat, -1.0)
        lqcd.lq_face_copy(H.h, bn, 2, H.h, an, 2, nat, 1.0)
        y = torch.empty((V, 4, 3), dtype=torch.complex128 if prec == lqcd.LQ_F64 else torch.complex64, device="cuda")
        lqcd.lq_convert(H.h, y, DT[prec], bn, nat)
        b = host(y).reshape(6, V3, 4, 3)
        ag = a.reshape(6, V3, 4, 3)
        # the same field after one round trip through the native format, for the FP16 rounding
        lqcd.lq_convert(H.h, y, DT[prec], an, nat)
        ar = host(y).reshape(6, V3, 4, 3)
    assert np.array_equal(b[4], -ar[1]) and np.array_equal(b[2], ar[2])
    assert not np.any(b[[0, 1, 3, 5]])
    assert rel_err(ar[1], ag[1]) < TOL[prec] * 2


def test_slices_and_face_copy_argument_checks():
    dims = (4, 4, 2, 4)
    U = inputs.gauge_field(dims, "unit")
    with Handle(dims, U) as H, Handle((4, 4, 4, 4), inputs.gauge_field((4, 4, 4, 4), "unit")) as H2:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        a, b = native_buffer(H.h, lqcd.LQ_F32), native_buffer(H.h, lqcd.LQ_F32)
        c = native_buffer(H2.h, lqcd.LQ_F32)
        for t0, t1 in ((0, 5), (2, 2), (-1, 2)):
            with pytest.raises(lqcd.LqError):
                lqcd.dslash_apply_slices(H.h, b, a, nat, t0, t1)
        with pytest.raises(lqcd.LqError):  # site-major fields
            lqcd.dslash_apply_slices(H.h, b, a, lqcd.LQ_F32, 0, 2)
        with pytest.raises(lqcd.LqError):  # L2 differs
            lqcd.lq_face_copy(H.h, a, 0, H2.h, c, 1, nat)
        with pytest.raises(lqcd.LqError):  # slice out of range
            lqcd.lq_face_copy(H.h, a, 4, H.h, b, 0, nat)
        with pytest.raises(lqcd.LqError):  # a slice onto itself
            lqcd.lq_face_copy(H.h, a, 1, H.h, a, 1, nat)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("sign", [1, -1])
def test_projected_face_wire_layout_and_ghost(prec, sign):
    """The wire holds scale * (psi_up + S psi_dn) per spatial parity in the
    slice's run order (checked element by element in FP64/FP32); its size is
    half the spinor's (plus the FP32 norm in FP16/BF16); the rebuilt ghost
    projects back to the same h through (1 + S gamma_t) and to zero through
    (1 - S gamma_t)."""
    dims = (4, 2, 6, 6)
    L0, L1, L2, L3 = dims
    V3 = L0 * L1 * L2
    n = V3 // 2
    a = inputs.gaussian_spinor(V3 * L3, seed=2203)
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        nat = lqcd.LQ_NATIVE | prec
        dt = DT.get(prec, lqcd.LQ_F32)
        an, bn = native_buffer(H.h, prec), native_buffer(H.h, prec)
        lqcd.lq_convert(H.h, an, nat, dev(a, dt), dt)
        lqcd.lq_convert(H.h, bn, nat, dev(np.zeros_like(a), dt), dt)
        nb = lqcd.lq_face_wire_bytes(H.h, nat)
        site = {lqcd.LQ_F64: 96, lqcd.LQ_F32: 48, lqcd.LQ_F16: 28, lqcd.LQ_BF16: 28}[prec]
        assert nb == 2 * n * site
        w = torch.empty(nb, dtype=torch.uint8, device="cuda")
        lqcd.lq_face_pack(H.h, w, an, 3, nat, sign, -1.0)
        lqcd.lq_face_unpack(H.h, bn, 2, w, nat, sign)  # an even distance: parity blocks stay
        lqcd.lq_face_unpack(H.h, bn, 5, w, nat, sign)  # an odd distance: parity blocks swap
        torch.cuda.synchronize()
        y = torch.empty((V3 * L3, 4, 3), dtype=torch.complex128 if prec == lqcd.LQ_F64 else torch.complex64,
                        device="cuda")
        lqcd.lq_convert(H.h, y, dt, an, nat)
        ar = host(y).reshape(L3, V3, 4, 3)  # the input after its round trip through the native format
        lqcd.lq_convert(H.h, y, dt, bn, nat)
        b = host(y).reshape(L3, V3, 4, 3)
        wh = w.cpu().numpy()
    ct = np.complex128 if prec == lqcd.LQ_F64 else np.complex64
    a3 = ar[3].astype(ct)  # exact: the values were stored in this precision (or narrower)
    h = -(a3[:, 0:2] + ct(sign) * a3[:, 2:4])  # the sum rounded as the kernel rounds it; scale -1
    x = coords3(dims[:3])
    sp = x.sum(axis=1) % 2
    if prec in (lqcd.LQ_F64, lqcd.LQ_F32):
        per = 1 if prec == lqcd.LQ_F64 else 2  # complex numbers per 16-byte plane element
        wv = wh.view(ct).reshape(2, 6 // per, n, per)  # [sp][plane][site][complex in plane]
        got = np.moveaxis(wv, 2, 1).reshape(2, n, 6)
        for q in (0, 1):
            assert np.array_equal(got[q], h[sp == q].reshape(n, 6).astype(ct))
    tol = 1e-15 if prec == lqcd.LQ_F64 else 1e-6 if prec == lqcd.LQ_F32 else 1e-2
    for t in (2, 5):
        g = b[t]
        proj = g[:, 0:2] + sign * g[:, 2:4]
        assert rel_err(proj, h) < tol
        assert np.max(np.abs(g[:, 0:2] - sign * g[:, 2:4])) <= tol * np.max(np.abs(h))
    assert not np.any(b[[0, 1, 3, 4]])


def coords3(d):
    L0, L1, L2 = d
    x2, x1, x0 = np.meshgrid(np.arange(L2), np.arange(L1), np.arange(L0), indexing="ij")
    return np.stack([x0.ravel(), x1.ravel(), x2.ravel()], axis=1)


def test_projected_face_argument_checks():
    dims = (4, 4, 2, 4)
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        a = native_buffer(H.h, lqcd.LQ_F32)
        w = torch.empty(lqcd.lq_face_wire_bytes(H.h, nat), dtype=torch.uint8, device="cuda")
        for args in ((a, 0, lqcd.LQ_F32, 1), (a, 0, nat, 0), (a, 4, nat, 1), (a, -1, nat, -1)):
            with pytest.raises(lqcd.LqError):
                lqcd.lq_face_pack(H.h, w, args[0], args[1], args[2], args[3])
            with pytest.raises(lqcd.LqError):
                lqcd.lq_face_unpack(H.h, args[0], args[1], w, args[2], args[3])
        with pytest.raises(lqcd.LqError):  # the wire inside the field
            lqcd.lq_face_pack(H.h, a[16:], a, 0, nat, 1)

