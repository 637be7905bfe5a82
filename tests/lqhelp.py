"""Helpers shared by the GPU parity tests: moving numpy fields to the device
and back, handle construction, and the comparison metrics."""
import numpy as np
import torch

from paper_2001_07557_gb300 import build as lqbuild
from paper_2001_07557_gb300 import lqcd

_built = False


def ensure_built():
    global _built
    if not _built:
        lqbuild.build()
        _built = True


def dev(a, prec=lqcd.LQ_F64):
    """numpy complex field -> contiguous CUDA tensor (complex128 or complex64)."""
    dt = np.complex128 if prec == lqcd.LQ_F64 else np.complex64
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def native_buffer(h, prec, subset=lqcd.LQ_FULL, nrhs=1, five_d=False):
    n = lqcd.lq_field_bytes(h, prec | lqcd.LQ_NATIVE, subset, nrhs, five_d)
    return torch.empty(n, dtype=torch.uint8, device="cuda")


class Handle:
    def __init__(self, dims, U, mass=0.1, bc=(1, 1, 1, -1), Ls=0, M5=0.0, mf=0.0, compress12=False,
                 U_prec=lqcd.LQ_F64, **kw):
        ensure_built()
        self.dims = dims
        self.params = lqcd.make_params(dims, bc=bc, mass=mass, Ls=Ls, M5=M5, mf=mf, compress12=compress12, **kw)
        self.U = dev(U, U_prec)
        self.h = lqcd.lq_create(self.params, self.U, U_prec)

    def close(self):
        if self.h:
            lqcd.lq_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def rel_err(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def max_err(a, b):
    """Largest element-wise error relative to the largest reference element."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
