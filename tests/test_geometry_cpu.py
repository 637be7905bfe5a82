"""CPU checks of the kernels' index arithmetic (replicated here in Python):
the multiply-shift division used for checkerboard coordinates, and the
neighbour checkerboard indices the hop kernel computes without tables."""
import numpy as np
import pytest


def div_magic(d):
    return (1 << 40) // d + 1


def fast_div(n, m):
    return (n * m) >> 40


@pytest.mark.parametrize("d", list(range(1, 70)) + [96, 127, 128, 255, 1000, 4095, 4096, 8191, 8192])
def test_fast_division_is_exact_below_2_27(d):
    m = div_magic(d)
    top = (1 << 27) - 1
    ns = set(range(0, 4000)) | {top, top - 1} | set(range(max(0, top - 3 * d), top + 1, max(1, d // 7)))
    ns |= {k * d + r for k in (1, 7, 12345, top // d - 1) for r in (-1, 0, 1) if 0 <= k * d + r <= top}
    for n in ns:
        assert fast_div(n, m) == n // d, (n, d)


def cb_coords(L, cb, p):
    Lh0 = L[0] // 2
    t1 = fast_div(cb, div_magic(Lh0))
    xh = cb - t1 * Lh0
    t2 = fast_div(t1, div_magic(L[1]))
    x1 = t1 - t2 * L[1]
    x3 = fast_div(t2, div_magic(L[2]))
    x2 = t2 - x3 * L[2]
    x0 = 2 * xh + ((p + x1 + x2 + x3) & 1)
    return [x0, x1, x2, x3]


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 6, 2, 8), (6, 4, 4, 2), (8, 2, 6, 4), (4, 4, 2, 4), (10, 4, 6, 2)])
def test_neighbour_indices_match_brute_force(L):
    V = int(np.prod(L))
    Vh = V // 2
    Lh0 = L[0] // 2

    def lexi(x):
        return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))

    for p in (0, 1):
        for i in range(Vh):
            x = cb_coords(L, i, p)
            assert lexi(x) // 2 == i and sum(x) % 2 == p
            xh = x[0] >> 1
            xf, xb = x[0] + 1, x[0] - 1
            if xf == L[0]:
                xf = 0
            if xb < 0:
                xb = L[0] - 1
            nf, nb = [i - xh + (xf >> 1)], [i - xh + (xb >> 1)]
            step = Lh0
            for mu in (1, 2, 3):
                top, bot = x[mu] == L[mu] - 1, x[mu] == 0
                nf.append(i - (L[mu] - 1) * step if top else i + step)
                nb.append(i + (L[mu] - 1) * step if bot else i - step)
                step *= L[mu]
            for mu in range(4):
                y = list(x)
                y[mu] = (y[mu] + 1) % L[mu]
                assert lexi(y) // 2 == nf[mu] and 0 <= nf[mu] < Vh
                y = list(x)
                y[mu] = (y[mu] - 1) % L[mu]
                assert lexi(y) // 2 == nb[mu] and 0 <= nb[mu] < Vh
