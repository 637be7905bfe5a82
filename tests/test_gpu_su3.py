"""GPU parity: the lattice-wide SU(3) product lq_su3_mul (the paper's
matrix-matrix benchmark, Sec. 3.3, Fig. 4a-c) against the FP64 oracle.

Tolerances, from the arithmetic of one entry (3 complex products summed):
FP64 1e-14 and FP32 2e-6 of the largest entry (inputs rounded to FP32 once,
then ~6 rounded operations per entry).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from lqhelp import ensure_built
from paper_2001_07557_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQ_F64: 1e-14, lqcd.LQ_F32: 2e-6}
DT = {lqcd.LQ_F64: (np.complex128, torch.complex128), lqcd.LQ_F32: (np.complex64, torch.complex64)}


def matrices(n, seed, kind="gauss"):
    if kind == "su3":
        L = max(1, int(np.ceil((n / 4) ** 0.25)))
        U = inputs.gauge_field((L, L, L, L), "random", seed=seed).reshape(-1, 3, 3)
        reps = int(np.ceil(n / len(U)))
        return np.ascontiguousarray(np.tile(U, (reps, 1, 1))[:n])
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))


def run(A, B, fmt, out=None):
    npd, tdt = DT[fmt]
    a = torch.from_numpy(A.astype(npd)).cuda()
    b = torch.from_numpy(B.astype(npd)).cuda()
    c = torch.empty_like(a) if out is None else out(a, b)
    lqcd.lq_su3_mul(c, a, b, len(A), fmt)
    torch.cuda.synchronize()
    return c.cpu().numpy().astype(np.complex128)


def check(got, want, fmt):
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= TOL[fmt], err


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    lqcd.lq_wait_timeouts()  # start from zero
    yield
    assert lqcd.lq_wait_timeouts() == 0


@pytest.mark.parametrize("fmt", [lqcd.LQ_F64, lqcd.LQ_F32])
@pytest.mark.parametrize("n", [1, 2, 3, 127, 128, 129, 255, 256, 257, 513, 4099, 100003])
def test_su3_mul_sizes(fmt, n):
    """Whole tiles, ragged last tiles (odd FP32 counts take the plain-load
    path for their last matrix) and more tiles than resident blocks."""
    A, B = matrices(n, 11), matrices(n, 12)
    want = oracle.su3_mul(A.astype(DT[fmt][0]), B.astype(DT[fmt][0]))
    check(run(A, B, fmt), want, fmt)


@pytest.mark.parametrize("fmt", [lqcd.LQ_F64, lqcd.LQ_F32])
def test_su3_mul_group_elements_and_in_place(fmt):
    """Random SU(3) factors (the benchmark's inputs) and C = A or C = B in place."""
    n = 3001
    A, B = matrices(n, 21, "su3"), matrices(n, 22, "su3")
    want = oracle.su3_mul(A.astype(DT[fmt][0]), B.astype(DT[fmt][0]))
    check(run(A, B, fmt), want, fmt)
    check(run(A, B, fmt, out=lambda a, b: a), want, fmt)
    check(run(A, B, fmt, out=lambda a, b: b), want, fmt)
    P = run(A, B, lqcd.LQ_F64) if fmt == lqcd.LQ_F64 else None
    if P is not None:
        assert np.max(np.abs(np.conj(np.swapaxes(P, 1, 2)) @ P - np.eye(3))) < 1e-13


@pytest.mark.slow
@pytest.mark.parametrize("fmt", [lqcd.LQ_F64, lqcd.LQ_F32])
def test_su3_mul_full_size(fmt):
    """The benchmark's size: 32^4 x 4 link matrices (4,194,304 products)."""
    n = 4 * 32 ** 4
    A, B = matrices(n, 31), matrices(n, 32)
    want = oracle.su3_mul(A.astype(DT[fmt][0]), B.astype(DT[fmt][0]))
    check(run(A, B, fmt), want, fmt)


def test_a_wait_that_runs_out_is_reported_and_the_device_stays_usable():
    """The failure path of the barrier waits, without a fault: a product tile
    whose barrier is armed for bytes that never come gives up after about a
    second, the count of waits that ran out reads 1, and the next product on
    the same context is correct."""
    import time

    assert lqcd.lq_wait_timeouts() == 0
    t0 = time.perf_counter()
    lqcd.lq_test_stalled_wait()
    dt = time.perf_counter() - t0
    # the synchronising read reports the wait that ran out as LQ_ERR_TIMEOUT, with the count
    count = ctypes.c_uint(0)
    assert lqcd.lib().lq_wait_timeouts(ctypes.byref(count)) == -7
    assert count.value == 1
    assert lqcd.lib().lq_wait_timeouts(ctypes.byref(count)) == 0 and count.value == 0
    assert 0.5 < dt < 20.0, dt
    A, B = matrices(1000, 41), matrices(1000, 42)
    check(run(A, B, lqcd.LQ_F32), oracle.su3_mul(A.astype(np.complex64), B.astype(np.complex64)), lqcd.LQ_F32)
