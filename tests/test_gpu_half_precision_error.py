"""Where the error of the 16-bit hops comes from.

The FP16/BF16 hop stores spinors as 16-bit values with an FP32 norm per site
and links as 16-bit values; its products and all colour, direction and
diagonal sums are FP32 (mixed-precision FMA on 16-bit inputs), but the spin
projection h = psi_up +- A psi_dn is one packed 16-bit addition, rounded once
like the stored inputs.  This test splits the hop's error against the FP64
oracle, on the same seeded inputs:

  e_store: the oracle's FP64 hop applied to the inputs rounded to the storage
           format (16-bit components of the site-normed spinor, 16-bit link
           entries), with its output rounded to the storage format as well;
  e_total: the GPU hop against the exact result.

Both carry the same rounding of the inputs and of the output; what the
kernel's own arithmetic (the 16-bit projection and the FP32 sums) adds is
independent of it, so e_extra = sqrt(e_total^2 - e_store^2).  The projection
rounds once, like one storage rounding of its inputs, so e_extra must stay
below e_store, i.e. e_total < sqrt(2) e_store: the hop's accuracy is set by its
storage format.  (Comparing the GPU output with the storage-only result
directly would mostly measure the two independent roundings of the output.)
"""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, native_buffer, rel_err
from paper_2001_07557_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu


def round16(x, prec):
    """Round float32 values to FP16 / BF16 (round to nearest even) and back; torch
    provides the BF16 rounding, which numpy lacks."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    dt = torch.float16 if prec == lqcd.LQ_F16 else torch.bfloat16
    return t.to(dt).to(torch.float32).numpy().astype(np.float64)


def store_spinor(psi, prec):
    """The native 16-bit spinor format: per-site FP32 norm = max |real component|,
    components divided by it in FP32 and rounded to 16 bits."""
    re = np.stack([psi.real, psi.imag], axis=-1).reshape(psi.shape[0], -1).astype(np.float32)
    nrm = np.max(np.abs(re), axis=1).astype(np.float32)
    inv = np.where(nrm > 0, np.float32(1) / np.where(nrm > 0, nrm, 1), 0).astype(np.float32)
    q = round16(re * inv[:, None], prec) * nrm[:, None].astype(np.float64)
    q = q.reshape(psi.shape + (2,))
    return q[..., 0] + 1j * q[..., 1]


def store_links(U, prec):
    q = round16(np.stack([U.real, U.imag], axis=-1).astype(np.float32), prec)
    return q[..., 0] + 1j * q[..., 1]


@pytest.mark.parametrize("prec", [lqcd.LQ_F16, lqcd.LQ_BF16])
@pytest.mark.parametrize("dag", [False, True])
def test_arithmetic_adds_less_than_storage(prec, dag):
    dims = (8, 8, 8, 8)
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1002)
    psi = inputs.gaussian_spinor(V // 2, seed=2002)
    exact = oracle.wilson_hop_eo(psi, U, dims, 0, dagger=dag)
    stored = store_spinor(oracle.wilson_hop_eo(store_spinor(psi, prec), store_links(U, prec), dims, 0,
                                               dagger=dag), prec)
    with Handle(dims, U) as H:
        nat = lqcd.LQ_NATIVE | prec
        xn = native_buffer(H.h, prec, lqcd.LQ_ODD)
        yn = native_buffer(H.h, prec, lqcd.LQ_EVEN)
        lqcd.lq_convert(H.h, xn, nat, dev(psi), lqcd.LQ_F64, lqcd.LQ_ODD)
        (lqcd.dslash_dag_apply if dag else lqcd.dslash_apply)(H.h, yn, xn, nat, lqcd.LQ_EVEN)
        y = torch.empty_like(dev(psi))
        lqcd.lq_convert(H.h, y, lqcd.LQ_F64, yn, nat, lqcd.LQ_EVEN)
        got = host(y) / -0.5  # dslash_apply(LQ_EVEN) returns -1/2 H_eo
    e_store = rel_err(stored, exact)
    e_total = rel_err(got, exact)
    e_extra = np.sqrt(max(e_total ** 2 - e_store ** 2, 0.0))
    print(f"prec {prec} dag {dag}: e_store {e_store:.3e} e_total {e_total:.3e} e_extra {e_extra:.3e}")
    assert e_total < np.sqrt(2.0) * e_store, (e_total, e_store)
