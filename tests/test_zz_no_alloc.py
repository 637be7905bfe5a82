"""lq_dot_noalloc, the inner product for callers that cannot allocate device
memory (their own pool owns the budget, cudaMalloc's device synchronisation
is not acceptable, or a stream capture is in progress).  It must give what
lq_dot gives, call after call, while its scratch is a fixed device array.

Collected last on purpose; it passes alone in a fresh process and after the
other tests."""
import ctypes

import numpy as np
import pytest
import torch

from lqhelp import Handle, dev
from paper_2001_07557_gb300 import inputs
from paper_2001_07557_gb300 import lqcd

pytestmark = pytest.mark.gpu

# the tolerances of tests/test_gpu_blas.py (relative to the field norms)
TOL = {lqcd.LQ_F64: 1e-13, lqcd.LQ_F32: 1e-6}


def c_abi_call(fn, h, res, a, b, fmt, subset, nrhs, five_d=0):
    st = torch.cuda.current_stream().cuda_stream
    return fn(ctypes.c_void_p(h), ctypes.c_void_p(res.data_ptr()), ctypes.c_void_p(a.data_ptr()),
              ctypes.c_void_p(b.data_ptr()), fmt, subset, nrhs, five_d, ctypes.c_void_p(st))


@pytest.mark.parametrize("prec", [lqcd.LQ_F64, lqcd.LQ_F32])
def test_noalloc_dot_matches_lq_dot_twice(prec):
    dims = (4, 6, 4, 4)
    V = int(np.prod(dims))
    nrhs = 3
    L = lqcd.lib()
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        for call in range(2):
            a = dev(inputs.gaussian_spinor(V, seed=10 + call, nrhs=nrhs), prec)
            b = dev(inputs.gaussian_spinor(V, seed=20 + call, nrhs=nrhs), prec)
            ref = torch.empty(2 * nrhs, dtype=torch.float64, device="cuda")
            got = torch.full((2 * nrhs,), float("nan"), dtype=torch.float64, device="cuda")
            assert c_abi_call(L.lq_dot, H.h, ref, a, b, prec, lqcd.LQ_FULL, nrhs) == 0
            assert c_abi_call(L.lq_dot_noalloc, H.h, got, a, b, prec, lqcd.LQ_FULL, nrhs) == 0
            torch.cuda.synchronize()
            scale = (a.reshape(nrhs, -1).norm(dim=1) * b.reshape(nrhs, -1).norm(dim=1)).cpu().numpy()
            diff = np.abs((got - ref).cpu().numpy().reshape(nrhs, 2)).max(axis=1)
            assert np.all(diff <= TOL[prec] * scale), (call, diff / scale)


def test_noalloc_dot_native_five_d_and_size_limit():
    dims = (4, 4, 4, 4)
    Ls = 4
    V = int(np.prod(dims))
    L = lqcd.lib()
    with Handle(dims, inputs.gauge_field(dims, "unit"), Ls=Ls, M5=1.8) as H:
        fmt = lqcd.LQ_NATIVE | lqcd.LQ_F64
        nb = lqcd.lq_field_bytes(H.h, fmt, five_d=True)
        a = torch.empty(nb, dtype=torch.uint8, device="cuda")
        lqcd.lq_convert(H.h, a, fmt, dev(inputs.gaussian_spinor(V, seed=5, nrhs=Ls)), lqcd.LQ_F64, five_d=True)
        for _ in range(2):
            ref = torch.empty(2, dtype=torch.float64, device="cuda")
            got = torch.empty(2, dtype=torch.float64, device="cuda")
            assert c_abi_call(L.lq_dot, H.h, ref, a, a, fmt, lqcd.LQ_FULL, 1, 1) == 0
            assert c_abi_call(L.lq_dot_noalloc, H.h, got, a, a, fmt, lqcd.LQ_FULL, 1, 1) == 0
            torch.cuda.synchronize()
            assert abs(got[0].item() - ref[0].item()) <= TOL[lqcd.LQ_F64] * ref[0].item()
        # more right-hand sides than the fixed scratch holds: rejected, nothing launched
        n = lqcd.LQ_DOT_NOALLOC_MAX_RHS + 1
        x = dev(inputs.gaussian_spinor(V, seed=6, nrhs=n))
        res = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
        assert c_abi_call(L.lq_dot_noalloc, H.h, res, x, x, lqcd.LQ_F64, lqcd.LQ_FULL, n) == -1  # LQ_ERR_ARG
        torch.cuda.synchronize()
        assert torch.count_nonzero(res).item() == 0


def _pageable_access():
    """cudaDevAttrPageableMemoryAccess (88) of device 0, read through the toolkit's runtime."""
    rt = ctypes.CDLL("/usr/local/cuda/lib64/libcudart.so")
    v = ctypes.c_int(0)
    assert rt.cudaDeviceGetAttribute(ctypes.byref(v), 88, 0) == 0
    return v.value


def test_noalloc_dot_result_must_be_device_addressable():
    """The result may be pinned host memory (mapped into the device's address
    space); a pageable host buffer on a device that cannot read pageable memory
    is rejected before any launch (LQ_ERR_LAYOUT) and left untouched."""
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    L = lqcd.lib()
    with Handle(dims, inputs.gauge_field(dims, "unit")) as H:
        a = dev(inputs.gaussian_spinor(V, seed=31))
        ref = torch.empty(2, dtype=torch.float64, device="cuda")
        assert c_abi_call(L.lq_dot, H.h, ref, a, a, lqcd.LQ_F64, lqcd.LQ_FULL, 1) == 0
        pinned = torch.zeros(2, dtype=torch.float64).pin_memory()
        assert c_abi_call(L.lq_dot_noalloc, H.h, pinned, a, a, lqcd.LQ_F64, lqcd.LQ_FULL, 1) == 0
        torch.cuda.synchronize()
        assert abs(pinned[0].item() - ref[0].item()) <= TOL[lqcd.LQ_F64] * ref[0].item()
        if _pageable_access():
            return  # pageable memory is addressable on this device: nothing to reject
        buf = np.zeros(2, dtype=np.float64)
        st = torch.cuda.current_stream().cuda_stream
        rc = L.lq_dot_noalloc(ctypes.c_void_p(H.h), ctypes.c_void_p(buf.ctypes.data), ctypes.c_void_p(a.data_ptr()),
                              ctypes.c_void_p(a.data_ptr()), lqcd.LQ_F64, lqcd.LQ_FULL, 1, 0, ctypes.c_void_p(st))
        torch.cuda.synchronize()
        assert rc == -2 and not buf.any()
