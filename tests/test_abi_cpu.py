"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/lqcd.h declares, and its structs match the header's layout.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2001_07557_gb300 import build as lqbuild
from paper_2001_07557_gb300 import lqcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lqcd.h")


@pytest.fixture(scope="module")
def L():
    lqbuild.build()
    return lqcd.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(lqcd.EXPORTS)


def test_every_declared_symbol_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", lqcd.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    names = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for fn in declared_functions():
        assert fn in names, fn
        assert getattr(L, fn) is not None


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lqcd.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(lq_params), sizeof(lq_cg_params), sizeof(lq_cg_stats),'
                   ' offsetof(lq_params, compress12), offsetof(lq_cg_params, x0_is_guess));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(lqcd.lq_params), ctypes.sizeof(lqcd.lq_cg_params), ctypes.sizeof(lqcd.lq_cg_stats),
            lqcd.lq_params.compress12.offset, lqcd.lq_cg_params.x0_is_guess.offset]
    assert got == want


def test_status_strings(L):
    assert lqcd.lq_status_string(0) == "ok"
    assert lqcd.lq_status_string(-5) == "solver did not converge"
    assert lqcd.lq_status_string(12345) == "unknown status"


def test_null_arguments_are_rejected_before_any_launch(L):
    p = lqcd.make_params((4, 4, 4, 4))
    h = ctypes.c_void_p()
    assert L.lq_create(ctypes.byref(h), ctypes.byref(p), None, 0, None) == -1
    assert L.lq_create(None, ctypes.byref(p), None, 0, None) == -1
    assert L.dslash_apply(None, None, None, 0, -1, 1, None) == -1
    assert L.lq_destroy(None) == -1
    # the later entry points: a null handle or pointer is LQ_ERR_ARG before anything else
    assert L.dwf_schur_apply(None, None, None, 0, 0, None) == -1
    assert L.dwf_eo_prepare(None, None, None, 0, None) == -1
    assert L.dwf_eo_reconstruct(None, None, None, None, 0, None) == -1
    assert L.lq_set_hop_kernel(None, 0) == -1
    n = ctypes.c_size_t(0)
    assert L.lq_face_wire_bytes(None, 0x10 | 2, ctypes.byref(n)) == -1
    assert L.lq_face_pack(None, None, None, 0, 0x10 | 2, 1, 1.0, None) == -1
    assert L.lq_face_unpack(None, None, 0, None, 0x10 | 2, 1, None) == -1
    assert L.lq_index_faults(None, None, None) == -1


def test_su3_mul_argument_checks_before_any_launch(L):
    """lq_su3_mul rejects bad arguments before touching the device: the
    pointers below are never dereferenced."""
    A, B = 0x10000, 0x20000
    assert L.lq_su3_mul(0x30000, A, B, -1, 0, None) == -1  # n < 0
    assert L.lq_su3_mul(0x30000, A, B, 4, 2, None) == -1  # FP16 is not a product format
    assert L.lq_su3_mul(None, A, B, 4, 0, None) == -1
    assert L.lq_su3_mul(0x30000, None, B, 4, 1, None) == -1
    assert L.lq_su3_mul(0x30008, A, B, 4, 0, None) == -2  # C not 16-byte aligned
    assert L.lq_su3_mul(0x30000, A + 8, B, 4, 1, None) == -2
    assert L.lq_su3_mul(A + 16, A, B, 4, 0, None) == -1  # C overlaps A without being A
    assert L.lq_su3_mul(B - 16, A, B, 4, 1, None) == -1  # C's 288 bytes run into B
    assert L.lq_su3_mul(None, None, None, 0, 0, None) == 0  # n = 0 is a no-op
    assert L.lq_wait_timeouts(None) == -1
