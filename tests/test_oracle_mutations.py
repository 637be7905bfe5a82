"""Each plausible mistake, planted in a copy of the oracle source, fails a pin.

The copy is compiled on the CPU into a temporary library and the pins from
test_oracle_pins.py are run against it through oracle.swapped_library; every
mutant must be caught by at least one of the pins listed for it.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "wilson_oracle.c")

# (name, original text, planted text, pins that must fail)
MUTANTS = [
    ("gamma sign on the forward hop", "fwd[mu][a][b] = id - s * g[a][b];", "fwd[mu][a][b] = id + s * g[a][b];",
     ["free"]),
    ("no conjugate on the backward link", "cplx m = adj ? conj(M[j * COL + i]) : M[i * COL + j];",
     "cplx m = adj ? M[j * COL + i] : M[i * COL + j];", ["cov"]),
    ("transposed forward link", "cplx m = adj ? conj(M[j * COL + i]) : M[i * COL + j];",
     "cplx m = adj ? conj(M[j * COL + i]) : M[j * COL + i];", ["cov"]),
    ("backward link read at x instead of x-mu", "U + (ym * 4 + mu) * 9, 1,", "U + (site * 4 + mu) * 9, 1,",
     ["cov"]),
    ("boundary phase dropped on the forward hop", "if (y[mu] == d[mu]) { y[mu] = 0; eta = bc[mu]; }",
     "if (y[mu] == d[mu]) { y[mu] = 0; }", ["free"]),
    ("hop normalised by 1 instead of 1/2", "out[i] = a * in[i] - 0.5 * out[i];", "out[i] = a * in[i] - out[i];",
     ["free"]),
    ("diagonal m + 2r", "double a = mass + 4.0 * r;\n    for (long i = 0; i < n; ++i) out[i] = a * in[i] - 0.5",
     "double a = mass + 2.0 * r;\n    for (long i = 0; i < n; ++i) out[i] = a * in[i] - 0.5", ["free"]),
    ("Schur coefficient 1/(2a)", "out[i] = a * in[i] - out[i] / (4.0 * a);",
     "out[i] = a * in[i] - out[i] / (2.0 * a);", ["schur"]),
    ("dagger keeps the forward projector", "double s = dagger ? -1.0 : 1.0;", "double s = 1.0;", ["adj"]),
    ("domain-wall projectors swapped", "const cplx(*Pup)[4] = dagger ? (const cplx(*)[4])Pp : (const cplx(*)[4])Pm;",
     "const cplx(*Pup)[4] = dagger ? (const cplx(*)[4])Pm : (const cplx(*)[4])Pp;", ["dwf"]),
    ("domain-wall wall sign", "if (sp == Ls) { sp = 0; cp = mf; }", "if (sp == Ls) { sp = 0; cp = -mf; }",
     ["dwf"]),
    ("CG beta inverted", "double beta = rr_new / rr;", "double beta = rr / rr_new;", ["cg"]),
    ("Moebius c5 term applied without the shift", "for (long i = 0; i < n5; ++i) u[i] = b5 * in[i] + c5 * t[i];",
     "for (long i = 0; i < n5; ++i) u[i] = b5 * in[i] + c5 * in[i];", ["mobius"]),
    ("Moebius dagger with the shift after the hop's b5 part", "for (long i = 0; i < n5; ++i) u[i] = c5 * t[i] - in[i];",
     "for (long i = 0; i < n5; ++i) u[i] = (c5 + b5) * t[i] - in[i];", ["mobius"]),
    ("domain-wall Schur complement sign", "for (long i = 0; i < n5; ++i) out[i] -= t[i];",
     "for (long i = 0; i < n5; ++i) out[i] += t[i];", ["dwf_eo"]),
    ("domain-wall M5 inverse ignores the dagger", "op(col, e, 1, Ls, prm, dagger);", "op(col, e, 1, Ls, prm, 0);",
     ["dwf_eo"]),
    ("domain-wall source preparation with the wrong sign", "for (long i = 0; i < n5; ++i) bhat[i] -= eo[i];",
     "for (long i = 0; i < n5; ++i) bhat[i] += eo[i];", ["dwf_eo"]),
    ("Moebius M5_M with the shift's sign flipped",
     "out[i] = (4.0 - M5) * (b5 * in[i] + c5 * out[i]) + in[i] - out[i];",
     "out[i] = (4.0 - M5) * (b5 * in[i] + c5 * out[i]) + in[i] + out[i];", ["mobius_eo"]),
    ("Moebius Schur complement with B^dag in M_oe", "mobius_b(u, in, Vh, Ls, mf, b5, c5, 0);",
     "mobius_b(u, in, Vh, Ls, mf, b5, c5, 1);", ["mobius_eo"]),
    ("Moebius source preparation without B", "mobius_b(eo, u, Vh, Ls, mf, b5, c5, 0);",
     "memcpy(eo, u, (size_t)n5 * sizeof(cplx));", ["mobius_eo"]),
    ("Moebius reconstruction with the wrong sign", "for (long i = 0; i < n5; ++i) eo[i] -= u[i];",
     "for (long i = 0; i < n5; ++i) eo[i] += u[i];", ["mobius_eo"]),
    ("SU(3) product with B transposed", "t += a[3 * i + k] * b[3 * k + j];", "t += a[3 * i + k] * b[3 * j + k];",
     ["su3"]),
    ("SU(3) product in the wrong order", "t += a[3 * i + k] * b[3 * k + j];", "t += b[3 * i + k] * a[3 * k + j];",
     ["su3"]),
]


def run_pin(kind, orc):
    if kind == "free":
        for dims, bc in [((4, 6, 2, 8), pins.BC_T), ((6, 4, 4, 2), (-1, 1, 1, 1))]:
            pins.test_free_field_closed_form(orc, dims, bc, 1.0)
    elif kind == "cov":
        pins.test_gauge_covariance(orc, (4, 4, 4, 4))
    elif kind == "adj":
        pins.test_dagger_is_adjoint_and_gamma5_hermitian(orc, (4, 4, 4, 4))
    elif kind == "schur":
        pins.test_even_odd_schur_solve_matches_full_solve(orc)
    elif kind == "dwf":
        pins.test_dwf_free_field_closed_form(orc)
    elif kind == "cg":
        pins.test_cg_matches_dense_lu_on_4444(orc)
    elif kind == "mobius":
        pins.test_mobius_reduces_to_shamir_and_its_c5_term_is_dw_times_s(orc)
    elif kind == "dwf_eo":
        pins.test_dwf_eo_schur_solve_matches_full_solve(orc)
    elif kind == "mobius_eo":
        pins.test_mobius_m5_is_the_zero_link_operator(orc)
        pins.test_mobius_eo_schur_solve_matches_full_solve(orc)
    elif kind == "su3":
        pins.test_su3_mul_matches_numpy_and_group_closure(orc)


@pytest.mark.parametrize("name,old,new,kinds", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, orc, name, old, new, kinds):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mutated = src.replace(old, new, 1)
    cfile = tmp_path / "mutant.c"
    cfile.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(cfile), "-o", str(so), "-lm"],
                   check=True)
    with oracle.swapped_library(str(so)):
        caught = False
        for kind in kinds:
            try:
                run_pin(kind, orc)
            except (AssertionError, np.linalg.LinAlgError):
                caught = True
        assert caught, f"no pin caught the planted mistake: {name}"
