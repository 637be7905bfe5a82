"""lq_dot: FP64-accumulated complex inner products against numpy."""
import numpy as np
import pytest
import torch

from lqhelp import Handle, dev, host
from paper_2001_07557_gb300 import inputs
from paper_2001_07557_gb300 import lqcd

pytestmark = pytest.mark.gpu


def want_dot(a, b, nrhs):
    a = a.reshape(nrhs, -1)
    b = b.reshape(nrhs, -1)
    return np.array([np.vdot(a[k], b[k]) for k in range(nrhs)])


def got_dot(res):
    r = res.cpu().numpy()
    return r[0::2] + 1j * r[1::2]


@pytest.mark.parametrize("subset", [lqcd.LQ_FULL, lqcd.LQ_EVEN])
@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
def test_dot_site_major(subset, prec):
    dims = (4, 6, 4, 2)
    V = int(np.prod(dims))
    n = V if subset == lqcd.LQ_FULL else V // 2
    a = inputs.gaussian_spinor(n, seed=1, nrhs=3)
    b = inputs.gaussian_spinor(n, seed=2, nrhs=3)
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        ad, bd = dev(a, prec), dev(b, prec)
        res = torch.empty(6, dtype=torch.float64, device="cuda")
        lqcd.lq_dot(H.h, res, ad, bd, prec, subset, nrhs=3)
        want = want_dot(host(ad), host(bd), 3)
        tol = 1e-13 if prec == lqcd.LQ_F64 else 1e-6
        assert np.max(np.abs(got_dot(res) - want) / np.abs(want)) < tol
        # repeated calls are bit-identical
        res2 = torch.empty_like(res)
        lqcd.lq_dot(H.h, res2, ad, bd, prec, subset, nrhs=3)
        assert torch.equal(res, res2)


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16, lqcd.LQ_BF16])
def test_dot_native_and_five_d(prec):
    dims = (4, 4, 4, 4)
    Ls = 3
    V = int(np.prod(dims))
    a = inputs.gaussian_spinor(V, seed=3, nrhs=Ls)
    b = inputs.gaussian_spinor(V, seed=4, nrhs=Ls)
    with Handle(dims, inputs.gauge_field(dims, "unit"), Ls=Ls, M5=1.8) as H:
        fmt = lqcd.LQ_NATIVE | prec
        nb = lqcd.lq_field_bytes(H.h, fmt, five_d=True)
        an = torch.empty(nb, dtype=torch.uint8, device="cuda")
        bn = torch.empty(nb, dtype=torch.uint8, device="cuda")
        lqcd.lq_convert(H.h, an, fmt, dev(a), lqcd.LQ_F64, five_d=True)
        lqcd.lq_convert(H.h, bn, fmt, dev(b), lqcd.LQ_F64, five_d=True)
        # the values as stored, read back in FP64
        a2 = torch.empty(Ls, V, 4, 3, dtype=torch.complex128, device="cuda")
        b2 = torch.empty_like(a2)
        lqcd.lq_convert(H.h, a2, lqcd.LQ_F64, an, fmt, five_d=True)
        lqcd.lq_convert(H.h, b2, lqcd.LQ_F64, bn, fmt, five_d=True)
        res = torch.empty(2, dtype=torch.float64, device="cuda")
        lqcd.lq_dot(H.h, res, an, bn, fmt, five_d=True)
        want = want_dot(host(a2), host(b2), 1)
        tol = 1e-13 if prec == lqcd.LQ_F64 else 1e-5
        assert abs(got_dot(res)[0] - want[0]) / np.linalg.norm(host(a2)) / np.linalg.norm(host(b2)) < tol
        # norm of a field: real and positive
        lqcd.lq_dot(H.h, res, an, an, fmt, five_d=True)
        r = got_dot(res)[0]
        assert abs(r.imag) < 1e-6 * r.real and abs(r.real - np.linalg.norm(host(a2)) ** 2) < tol * r.real


def test_dot_argument_checks():
    dims = (4, 4, 4, 4)
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        a = dev(inputs.gaussian_spinor(256, seed=1))
        res = torch.empty(2, dtype=torch.float64, device="cuda")
        L = lqcd.lib()
        st = torch.cuda.current_stream().cuda_stream
        assert L.lq_dot(H.h, None, a.data_ptr(), a.data_ptr(), 0, -1, 1, 0, st) == -1
        assert L.lq_dot(H.h, res.data_ptr(), a.data_ptr() + 8, a.data_ptr(), 0, -1, 1, 0, st) == -2
        assert L.lq_dot(H.h, res.data_ptr(), a.data_ptr(), a.data_ptr(), 0, -1, 0, 0, st) == -1
        assert L.lq_dot(H.h, res.data_ptr(), a.data_ptr(), a.data_ptr(), 0, -1, 1, 1, st) == -1  # Ls = 0
