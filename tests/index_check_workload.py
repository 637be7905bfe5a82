"""Workload of the index-checked build test (run as a script, with LQCD_LIBRARY
naming liblqcd_checked.so): the hop kernels in every storage precision and
shape they have -- full lattice, one parity, Schur complement, dagger, several
right-hand sides (CUDA cores and tensor cores), domain wall (Shamir and Moebius,
full and even-odd), a range of time slices, the uneven batch and a mixed CG --
on small lattices with ragged tiles and antiperiodic directions, each result
compared with the FP64 oracle.  Prints one JSON line: the index record of
lq_index_faults and the largest relative error per kind of launch."""
import json
import os
import sys

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[:0] = [_HERE, os.path.dirname(_HERE)]  # tests/ (lqhelp) and the repository root (oracle, package)

import oracle  # noqa: E402
from lqhelp import Handle, dev, host, native_buffer, rel_err  # noqa: E402
from paper_2001_07557_gb300 import inputs, lqcd  # noqa: E402

DT = {lqcd.LQ_F64: lqcd.LQ_F64, lqcd.LQ_F32: lqcd.LQ_F32, lqcd.LQ_F16: lqcd.LQ_F32, lqcd.LQ_BF16: lqcd.LQ_F32}
errors = {}
launches = 0


def note(kind, got, want):
    global launches
    launches += 1
    errors[kind] = max(errors.get(kind, 0.0), rel_err(got, want))


def native_apply(H, prec, psi, parity, nrhs, dag, sub_in, sub_out):
    nat = lqcd.LQ_NATIVE | prec
    x = dev(psi, DT[prec])
    xn, yn = native_buffer(H.h, prec, sub_in, nrhs), native_buffer(H.h, prec, sub_out, nrhs)
    lqcd.lq_convert(H.h, xn, nat, x, DT[prec], sub_in, nrhs)
    (lqcd.dslash_dag_apply if dag else lqcd.dslash_apply)(H.h, yn, xn, nat, parity, nrhs)
    y = torch.empty_like(x)
    lqcd.lq_convert(H.h, y, DT[prec], yn, nat, sub_out, nrhs)
    return host(y)


def wilson(dims, bc, m=0.07):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=1501)
    for prec in (lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16, lqcd.LQ_BF16):
        for nrhs in (1, 3):
            psi = inputs.gaussian_spinor(V, seed=2501, nrhs=nrhs)
            half = inputs.to_half(psi, dims, 0)
            with Handle(dims, U, mass=m, bc=bc) as H:
                for dag in (False, True):
                    got = native_apply(H, prec, psi, lqcd.LQ_FULL, nrhs, dag, lqcd.LQ_FULL, lqcd.LQ_FULL)
                    for k in range(nrhs):
                        note(f"full_p{prec}", got[k], oracle.wilson_dslash(psi[k], U, dims, m, bc=bc, dagger=dag))
                    got = native_apply(H, prec, half, lqcd.LQ_SCHUR_EVEN, nrhs, dag, lqcd.LQ_EVEN, lqcd.LQ_EVEN)
                    for k in range(nrhs):
                        note(f"schur_p{prec}", got[k], oracle.wilson_schur(half[k], U, dims, m, bc=bc, dagger=dag))
                    got = native_apply(H, prec, half, lqcd.LQ_ODD, nrhs, dag, lqcd.LQ_EVEN, lqcd.LQ_ODD)
                    for k in range(nrhs):
                        want = -0.5 * oracle.wilson_hop_eo(half[k], U, dims, lqcd.LQ_ODD, bc=bc, dagger=dag)
                        note(f"block_p{prec}", got[k], want)


def many_rhs(dims):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1502)
    psi = inputs.gaussian_spinor(V, seed=2502, nrhs=12)
    with Handle(dims, U, mass=0.05) as H:
        for kind in (lqcd.LQ_HOP_CUDA_CORES, lqcd.LQ_HOP_TENSOR_CORES):
            lqcd.lq_set_hop_kernel(H.h, kind)
            got = native_apply(H, lqcd.LQ_F16, psi, lqcd.LQ_FULL, 12, False, lqcd.LQ_FULL, lqcd.LQ_FULL)
            for k in range(12):
                note(f"rhs12_kind{kind}", got[k], oracle.wilson_dslash(psi[k], U, dims, 0.05))


def domain_wall(dims, Ls=3):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=1503)
    psi = inputs.gaussian_spinor(V, seed=2503, nrhs=Ls)
    pe = inputs.gaussian_spinor(V // 2, seed=2504, nrhs=Ls)
    for prec in (lqcd.LQ_F64, lqcd.LQ_F32, lqcd.LQ_F16):
        with Handle(dims, U, Ls=Ls, M5=1.8, mf=0.05) as H:
            x = dev(psi, DT[prec])
            y = torch.empty_like(x)
            if prec == lqcd.LQ_F16:
                nat = lqcd.LQ_NATIVE | prec
                xn, yn = (native_buffer(H.h, prec, five_d=True) for _ in range(2))
                lqcd.lq_convert(H.h, xn, nat, x, DT[prec], five_d=True)
                lqcd.dwf_dslash_apply(H.h, yn, xn, nat, False)
                lqcd.lq_convert(H.h, y, DT[prec], yn, nat, five_d=True)
            else:
                lqcd.dwf_dslash_apply(H.h, y, x, prec, False)
            note(f"dwf_p{prec}", host(y), oracle.dwf_dslash(psi, U, dims, Ls, 1.8, 0.05))
            if prec != lqcd.LQ_F16:
                xe = dev(pe, prec)
                ye = torch.empty_like(xe)
                lqcd.dwf_schur_apply(H.h, ye, xe, prec, True)
                note(f"dwf_schur_p{prec}", host(ye), oracle.dwf_schur(pe, U, dims, Ls, 1.8, 0.05, dagger=True))
    with Handle(dims, U, Ls=Ls, M5=1.8, mf=0.05, mobius=True, b5=1.5, c5=0.5) as H:
        xe = dev(pe)
        ye = torch.empty_like(xe)
        lqcd.dwf_schur_apply(H.h, ye, xe, lqcd.LQ_F64, False)
        note("mobius_schur", host(ye), oracle.dwf_mobius_schur(pe, U, dims, Ls, 1.8, 0.05, 1.5, 0.5))


def slices(dims):
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "random", seed=1504)
    psi = inputs.gaussian_spinor(V, seed=2505)
    with Handle(dims, U, mass=0.1) as H:
        nat = lqcd.LQ_NATIVE | lqcd.LQ_F32
        xn, yn = native_buffer(H.h, lqcd.LQ_F32), native_buffer(H.h, lqcd.LQ_F32)
        lqcd.lq_convert(H.h, xn, nat, dev(psi, lqcd.LQ_F32), lqcd.LQ_F32)
        lqcd.dslash_apply_slices(H.h, yn, xn, nat, 0, dims[3] // 2)
        lqcd.dslash_apply_slices(H.h, yn, xn, nat, dims[3] // 2, dims[3])
        y = torch.empty((V, 4, 3), dtype=torch.complex64, device="cuda")
        lqcd.lq_convert(H.h, y, lqcd.LQ_F32, yn, nat)
        note("slices", host(y), oracle.wilson_dslash(psi, U, dims, 0.1))


def solvers():
    dims, m = (4, 4, 2, 6), 0.1
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, "smooth", seed=1505)
    src = inputs.gaussian_spinor(V // 2, seed=2506, nrhs=4)
    with Handle(dims, U, mass=m) as H:
        b = dev(src)
        x = torch.zeros_like(b)
        cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_EO_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=4, tol=1e-10,
                                 inner=lqcd.LQ_F16)
        rc, st = lqcd.cg_solve(H.h, x, b, cp)
        assert rc == 0
        xs = host(x)
    prm = oracle.params(dims, mass=m)
    for k in range(4):
        note("cg_mixed_eo", oracle.apply_normal(oracle.OP_WILSON_EO, xs[k], U, prm), src[k])
    # the uneven batch: two lattices of different sizes in one persistent launch per step
    hs, xs_, bs_, Us = [], [], [], []
    for dims_l in ((4, 4, 2, 4), (6, 4, 2, 4)):
        Vl = int(np.prod(dims_l))
        Ul = inputs.gauge_field(dims_l, "smooth", seed=1506 + Vl)
        H = Handle(dims_l, Ul, mass=m)
        hs.append(H)
        Us.append((dims_l, Ul))
        bs_.append(dev(inputs.gaussian_spinor(Vl, seed=2507 + Vl, nrhs=2)))
        xs_.append(torch.zeros_like(bs_[-1]))
    cp = lqcd.make_cg_params(lqcd.LQ_OP_WILSON_NORMAL, lqcd.LQ_CG_MIXED, lqcd.LQ_F64, nrhs=2, tol=1e-10,
                             inner=lqcd.LQ_F16)
    rc, _ = lqcd.lq_batch_cg_solve([H.h for H in hs], xs_, bs_, cp)
    assert rc == 0
    for (dims_l, Ul), xb, bb in zip(Us, xs_, bs_):
        prm = oracle.params(dims_l, mass=m)
        for k in range(2):
            note("batch_cg", oracle.apply_normal(oracle.OP_WILSON, host(xb)[k], Ul, prm), host(bb)[k])
    for H in hs:
        H.close()


if __name__ == "__main__":
    for dims, bc in (((4, 6, 2, 8), (1, 1, 1, -1)), ((6, 2, 4, 2), (-1, 1, -1, 1))):
        wilson(dims, bc)
    many_rhs((6, 4, 2, 4))
    domain_wall((4, 2, 2, 6))
    slices((4, 4, 2, 8))
    solvers()
    count, first, checked = lqcd.lq_index_faults()
    print(json.dumps({"checked": checked, "faults": count, "first": first, "launches": launches,
                      "errors": errors}))
