"""lq_batch_cg_solve: independent lattices of different sizes in one
persistent, graph-captured solve, against the per-lattice solver and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from lqhelp import Handle, dev, host, rel_err
from paper_2001_07557_gb300 import inputs
from paper_2001_07557_gb300 import lqcd

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 6, 6, 6), (4, 4, 8, 8), (8, 8, 8, 8)]


@pytest.mark.parametrize("inner", [lqcd.LQ_F16, lqcd.LQ_BF16, lqcd.LQ_F32])
@pytest.mark.parametrize("op", [lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_OP_WILSON_NORMAL])
def test_uneven_batch_mixed(inner, op):
    nr = 3
    m = 0.05
    Hs, bs, xs, want = [], [], [], []
    try:
        for i, dims in enumerate(SHAPES):
            V = int(np.prod(dims))
            U = inputs.gauge_field(dims, "smooth", seed=1100 + i)
            n = V // 2 if op == lqcd.LQ_OP_WILSON_EO_NORMAL else V
            b = inputs.gaussian_spinor(n, seed=2100 + i, nrhs=nr)
            H = Handle(dims, U, mass=m)
            Hs.append(H)
            bs.append(dev(b))
            xs.append(torch.zeros_like(bs[-1]))
            prm = oracle.params(dims, mass=m)
            oop = oracle.OP_WILSON_EO if op == lqcd.LQ_OP_WILSON_EO_NORMAL else oracle.OP_WILSON
            want.append([oracle.cg(oop, b[k], U, prm, 1e-12)[0] for k in range(nr)])
        cp = lqcd.make_cg_params(op, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=nr, tol=1e-10, inner=inner)
        rc, st = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, cp)
        assert rc == 0
        for i in range(len(SHAPES)):
            xg = host(xs[i])
            for k in range(nr):
                assert st[i * nr + k].true_rel_residual < 1e-10
                assert rel_err(xg[k], want[i][k]) < 1e-7
        # a second solve reuses the tuned launch shape and gives the same answer
        xs2 = [torch.zeros_like(b) for b in bs]
        rc, st2 = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs2, bs, cp)
        assert rc == 0
        for i in range(len(SHAPES)):
            assert torch.allclose(xs2[i], xs[i], rtol=0, atol=1e-9 * float(xs[i].abs().max()))
    finally:
        for H in Hs:
            H.close()


def test_batch_plain_fp32_and_argument_checks():
    dims_list = [(4, 4, 4, 4), (4, 4, 4, 8)]
    Hs, bs, xs = [], [], []
    try:
        for i, dims in enumerate(dims_list):
            V = int(np.prod(dims))
            H = Handle(dims, inputs.gauge_field(dims, "smooth", seed=1200 + i), mass=0.1)
            Hs.append(H)
            bs.append(dev(inputs.gaussian_spinor(V // 2, seed=2200 + i, nrhs=2), lqcd.LQ_F32))
            xs.append(torch.zeros_like(bs[-1]))
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F32, nrhs=2, tol=1e-5)
        rc, st = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, cp)
        assert rc == 0 and all(s.status == 0 for s in st)
        # FP64 plain is not a batched mode; DWF is not batched; the same handle twice is refused
        for bad in (lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_PLAIN, lqcd.LQ_F64, nrhs=2),
                    lqcd.make_cg_params(lqcd.LQ_OP_DWF_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=2)):
            rc, _ = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, bad, check=False)
            assert rc == -1
        rc, _ = lqcd.lq_batch_cg_solve([Hs[0].h, Hs[0].h], xs, bs, cp, check=False)
        assert rc == -1
    finally:
        for H in Hs:
            H.close()


def test_uneven_batch_with_a_zero_right_hand_side():
    """One right-hand side of one lattice is zero: it is finished from the start
    (solution zero, no iterations), and the FP32 middle level of the others is
    unaffected."""
    nr, m = 2, 0.05
    Hs, bs, xs = [], [], []
    try:
        for i, dims in enumerate(SHAPES[:3]):
            V = int(np.prod(dims))
            U = inputs.gauge_field(dims, "smooth", seed=1150 + i)
            b = inputs.gaussian_spinor(V // 2, seed=2150 + i, nrhs=nr)
            if i == 1:
                b[0] = 0
            Hs.append(Handle(dims, U, mass=m))
            bs.append(dev(b))
            xs.append(torch.full_like(bs[-1], 3.0))
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=nr, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.lq_batch_cg_solve([H.h for H in Hs], xs, bs, cp)
        assert rc == 0
        assert np.all(host(xs[1])[0] == 0) and st[1 * nr + 0].iters == 0
        for g, s_ in enumerate(st):
            if g != nr:
                assert s_.true_rel_residual < 1e-10
    finally:
        for H in Hs:
            H.close()
