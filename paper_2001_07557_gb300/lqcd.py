"""Thin ctypes binding of liblqcd.so: the C entry points under the same names.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Field arguments are torch CUDA tensors (their data_ptr() is passed)
or raw integer device pointers; streams are torch.cuda.Stream objects, raw
cudaStream_t integers, or None for the current torch stream.  A non-zero
status raises LqError.  There is no CPU fallback: importing the binding
without a built liblqcd.so raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# LQCD_LIBRARY names another build of the same library (the index-checked
# liblqcd_checked.so of build.build(checked=True)); by default the in-tree build
LIB_PATH = os.environ.get("LQCD_LIBRARY") or os.path.join(_PKG, "liblqcd.so")

LQ_OK = 0
LQ_F64, LQ_F32, LQ_F16, LQ_BF16 = 0, 1, 2, 3
LQ_NATIVE = 0x10
LQ_FULL, LQ_EVEN, LQ_ODD, LQ_SCHUR_EVEN = -1, 0, 1, 2
LQ_OP_WILSON_NORMAL, LQ_OP_WILSON_EO_NORMAL, LQ_OP_DWF_NORMAL, LQ_OP_DWF_EO_NORMAL = 0, 1, 2, 3
LQ_CG_PLAIN, LQ_CG_MIXED, LQ_CG_BLOCK, LQ_CG_BATCHED = 0, 1, 2, 3
STATUS = {0: "LQ_OK", -1: "LQ_ERR_ARG", -2: "LQ_ERR_LAYOUT", -3: "LQ_ERR_CUDA", -4: "LQ_ERR_NOMEM",
          -5: "LQ_ERR_NOT_CONVERGED", -6: "LQ_ERR_BREAKDOWN", -7: "LQ_ERR_TIMEOUT", -8: "LQ_ERR_NAN"}

# every function the header declares
EXPORTS = ["lq_create", "lq_destroy", "lq_field_bytes", "lq_convert", "dslash_apply", "dslash_dag_apply",
           "lq_set_hop_kernel", "dwf_dslash_apply", "dwf_schur_apply", "dwf_eo_prepare", "dwf_eo_reconstruct", "lq_dot", "lq_dot_noalloc", "cg_solve", "lq_batch_cg_solve", "dslash_apply_slices",
           "lq_face_copy", "lq_face_wire_bytes", "lq_face_pack", "lq_face_unpack", "lq_su3_mul", "lq_wait_timeouts", "lq_test_stalled_wait", "lq_index_faults", "lq_status_string"]
LQ_DOT_NOALLOC_MAX_RHS = 32


class LqError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status})")


class lq_params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("bc", ctypes.c_int * 4), ("mass", ctypes.c_double),
                ("r", ctypes.c_double), ("Ls", ctypes.c_int), ("M5", ctypes.c_double), ("mf", ctypes.c_double),
                ("compress12", ctypes.c_int), ("mobius", ctypes.c_int), ("b5", ctypes.c_double),
                ("c5", ctypes.c_double)]


class lq_cg_params(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("mode", ctypes.c_int), ("fmt", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("inner", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("x0_is_guess", ctypes.c_int)]


class lq_cg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("status", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("time_ms", ctypes.c_double)]


_lib = None


def lib():
    """Load liblqcd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2001_07557_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.lq_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(lq_params), vp, i, vp]
        L.lq_destroy.argtypes = [vp]
        L.lq_field_bytes.argtypes = [vp, i, i, i, i, ctypes.POINTER(sz)]
        L.lq_convert.argtypes = [vp, vp, i, vp, i, i, i, i, vp]
        L.dslash_apply.argtypes = [vp, vp, vp, i, i, i, vp]
        L.dslash_dag_apply.argtypes = [vp, vp, vp, i, i, i, vp]
        L.dwf_dslash_apply.argtypes = [vp, vp, vp, i, i, vp]
        L.dwf_schur_apply.argtypes = [vp, vp, vp, i, i, vp]
        L.dwf_eo_prepare.argtypes = [vp, vp, vp, i, vp]
        L.dwf_eo_reconstruct.argtypes = [vp, vp, vp, vp, i, vp]
        L.lq_dot.argtypes = [vp, vp, vp, vp, i, i, i, i, vp]
        L.lq_dot_noalloc.argtypes = [vp, vp, vp, vp, i, i, i, i, vp]
        L.cg_solve.argtypes = [vp, vp, vp, ctypes.POINTER(lq_cg_params), ctypes.POINTER(lq_cg_stats), vp]
        L.lq_batch_cg_solve.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(lq_cg_params), ctypes.POINTER(lq_cg_stats), vp]
        L.dslash_apply_slices.argtypes = [vp, vp, vp, i, i, i, i, vp]
        L.lq_face_copy.argtypes = [vp, vp, i, vp, vp, i, i, ctypes.c_double, vp]
        L.lq_set_hop_kernel.argtypes = [vp, i]
        L.lq_index_faults.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(i)]
        L.lq_face_wire_bytes.argtypes = [vp, i, ctypes.POINTER(ctypes.c_size_t)]
        L.lq_face_pack.argtypes = [vp, vp, vp, i, i, i, ctypes.c_double, vp]
        L.lq_face_unpack.argtypes = [vp, vp, i, vp, i, i, vp]
        L.lq_su3_mul.argtypes = [vp, vp, vp, ctypes.c_long, i, vp]
        L.lq_wait_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint)]
        L.lq_test_stalled_wait.argtypes = []
        L.lq_status_string.argtypes = [i]
        L.lq_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "lq_status_string":
                getattr(L, name).restype = i
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s):
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, where):
    if rc != LQ_OK:
        raise LqError(rc, where)
    return rc


def make_params(dims, bc=(1, 1, 1, -1), mass=0.0, r=1.0, Ls=0, M5=0.0, mf=0.0, compress12=False, mobius=False,
                b5=1.0, c5=0.0) -> lq_params:
    p = lq_params()
    p.dims = (ctypes.c_int * 4)(*[int(d) for d in dims])
    p.bc = (ctypes.c_int * 4)(*[int(b) for b in bc])
    p.mass, p.r, p.Ls, p.M5, p.mf = float(mass), float(r), int(Ls), float(M5), float(mf)
    p.compress12 = int(bool(compress12))
    p.mobius, p.b5, p.c5 = int(bool(mobius)), float(b5), float(c5)
    return p


def lq_create(params: lq_params, U, U_prec=LQ_F64, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().lq_create(ctypes.byref(h), ctypes.byref(params), _ptr(U), U_prec, _stream(stream)), "lq_create")
    return h.value


def lq_destroy(h: int) -> None:
    _check(lib().lq_destroy(h), "lq_destroy")


def lq_field_bytes(h: int, fmt: int, subset: int = LQ_FULL, nrhs: int = 1, five_d: bool = False) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().lq_field_bytes(h, fmt, subset, nrhs, int(five_d), ctypes.byref(n)), "lq_field_bytes")
    return n.value


def lq_convert(h, dst, dst_fmt, src, src_fmt, subset=LQ_FULL, nrhs=1, five_d=False, stream=None):
    _check(lib().lq_convert(h, _ptr(dst), dst_fmt, _ptr(src), src_fmt, subset, nrhs, int(five_d), _stream(stream)),
           "lq_convert")


def dslash_apply(h, out, inp, fmt, parity=LQ_FULL, nrhs=1, stream=None):
    _check(lib().dslash_apply(h, _ptr(out), _ptr(inp), fmt, parity, nrhs, _stream(stream)), "dslash_apply")


def dslash_dag_apply(h, out, inp, fmt, parity=LQ_FULL, nrhs=1, stream=None):
    _check(lib().dslash_dag_apply(h, _ptr(out), _ptr(inp), fmt, parity, nrhs, _stream(stream)), "dslash_dag_apply")


def dwf_dslash_apply(h, out, inp, fmt, dagger=False, stream=None):
    _check(lib().dwf_dslash_apply(h, _ptr(out), _ptr(inp), fmt, int(dagger), _stream(stream)), "dwf_dslash_apply")


def dwf_schur_apply(h, out, inp, fmt, dagger=False, stream=None):
    """Even-odd domain-wall Schur complement Mhat (or Mhat^dag) on 5-d even half fields."""
    _check(lib().dwf_schur_apply(h, _ptr(out), _ptr(inp), fmt, int(dagger), _stream(stream)), "dwf_schur_apply")


def dwf_eo_prepare(h, bhat_e, eta, fmt, stream=None):
    """bhat_e = eta_e - M_eo M5^{-1} eta_o from a full 5-d source."""
    _check(lib().dwf_eo_prepare(h, _ptr(bhat_e), _ptr(eta), fmt, _stream(stream)), "dwf_eo_prepare")


def dwf_eo_reconstruct(h, psi, x_e, eta, fmt, stream=None):
    """The full 5-d solution from its even half and the source."""
    _check(lib().dwf_eo_reconstruct(h, _ptr(psi), _ptr(x_e), _ptr(eta), fmt, _stream(stream)),
           "dwf_eo_reconstruct")


def lq_dot(h, result, a, b, fmt, subset=LQ_FULL, nrhs=1, five_d=False, stream=None):
    """result: device float64 tensor of 2 * nrhs entries, (re, im) per right-hand side."""
    _check(lib().lq_dot(h, _ptr(result), _ptr(a), _ptr(b), fmt, subset, nrhs, int(five_d), _stream(stream)),
           "lq_dot")


def lq_dot_noalloc(h, result, a, b, fmt, subset=LQ_FULL, nrhs=1, five_d=False, stream=None):
    """lq_dot without any device allocation (scratch in a fixed device array);
    nrhs <= LQ_DOT_NOALLOC_MAX_RHS."""
    _check(lib().lq_dot_noalloc(h, _ptr(result), _ptr(a), _ptr(b), fmt, subset, nrhs, int(five_d),
                                _stream(stream)), "lq_dot_noalloc")


def make_cg_params(op, mode=LQ_CG_PLAIN, fmt=LQ_F64, nrhs=1, tol=1e-10, maxiter=100000, inner=LQ_F32,
                   inner_tol=0.0, x0_is_guess=False) -> lq_cg_params:
    c = lq_cg_params()
    c.op, c.mode, c.fmt, c.nrhs, c.tol, c.maxiter = int(op), int(mode), int(fmt), int(nrhs), float(tol), int(maxiter)
    c.inner, c.inner_tol, c.x0_is_guess = int(inner), float(inner_tol), int(bool(x0_is_guess))
    return c


def cg_solve(h, x, b, cp: lq_cg_params, stream=None, check=True):
    """Returns (status, [lq_cg_stats per right-hand side])."""
    stats = (lq_cg_stats * max(1, cp.nrhs))()
    rc = lib().cg_solve(h, _ptr(x), _ptr(b), ctypes.byref(cp), stats, _stream(stream))
    if check and rc not in (LQ_OK,):
        raise LqError(rc, "cg_solve")
    return rc, list(stats)


def lq_batch_cg_solve(hs, xs, bs, cp: lq_cg_params, stream=None, check=True):
    n = len(hs)
    H = (ctypes.c_void_p * n)(*hs)
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    B = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    stats = (lq_cg_stats * (n * max(1, cp.nrhs)))()
    rc = lib().lq_batch_cg_solve(H, n, X, B, ctypes.byref(cp), stats, _stream(stream))
    if check and rc != LQ_OK:
        raise LqError(rc, "lq_batch_cg_solve")
    return rc, list(stats)


def lq_status_string(status: int) -> str:
    return lib().lq_status_string(status).decode()


def lq_su3_mul(C, A, B, n, fmt, stream=None):
    """C[x] = A[x] B[x] for n 3x3 complex matrices [x][row][col]{re, im},
    fmt LQ_F64 or LQ_F32 (device pointers or tensors, 16-byte aligned)."""
    _check(lib().lq_su3_mul(_ptr(C), _ptr(A), _ptr(B), int(n), fmt, _stream(stream)), "lq_su3_mul")


def lq_wait_timeouts():
    """Device-side barrier waits that ran out since the last call (resets the count)."""
    c = ctypes.c_uint(0)
    rc = lib().lq_wait_timeouts(ctypes.byref(c))
    if rc != -7:  # LQ_ERR_TIMEOUT: the count is not zero (it is still returned)
        _check(rc, "lq_wait_timeouts")
    return c.value


def lq_test_stalled_wait():
    """Run one product tile whose barrier wait must run out (tests the timeout path)."""
    _check(lib().lq_test_stalled_wait(), "lq_test_stalled_wait")


def dslash_apply_slices(h, out, inp, fmt, t0, t1, dagger=False, stream=None):
    """Full-lattice D (or D^dag) on native fields with output on time slices [t0, t1) only."""
    _check(lib().dslash_apply_slices(h, _ptr(out), _ptr(inp), fmt, int(t0), int(t1), int(dagger), _stream(stream)),
           "dslash_apply_slices")


def lq_face_copy(hd, dst, t_dst, hs, src, t_src, fmt, scale=1.0, stream=None):
    """Time slice t_src of src (hs's lattice) times scale into slice t_dst of dst (hd's lattice)."""
    _check(lib().lq_face_copy(hd, _ptr(dst), int(t_dst), hs, _ptr(src), int(t_src), fmt, float(scale),
                              _stream(stream)), "lq_face_copy")


LQ_HOP_CUDA_CORES, LQ_HOP_TENSOR_CORES = 0, 1


def lq_set_hop_kernel(h, kind):
    """LQ_HOP_CUDA_CORES (default), or LQ_HOP_TENSOR_CORES: the tensor-core hop for launches of
    >= 8 FP16/BF16 right-hand sides with 18-real links."""
    _check(lib().lq_set_hop_kernel(h, int(kind)), "lq_set_hop_kernel")


def lq_index_faults():
    """(count, first, checked): out-of-range hop indices since the last call (index-checked build)."""
    c, f, k = ctypes.c_ulonglong(0), ctypes.c_longlong(-1), ctypes.c_int(0)
    _check(lib().lq_index_faults(ctypes.byref(c), ctypes.byref(f), ctypes.byref(k)), "lq_index_faults")
    return c.value, f.value, k.value


def lq_face_wire_bytes(h, fmt):
    """Bytes of one spin-projected face buffer of h's time slices in format fmt."""
    n = ctypes.c_size_t(0)
    _check(lib().lq_face_wire_bytes(h, fmt, ctypes.byref(n)), "lq_face_wire_bytes")
    return n.value


def lq_face_pack(h, wire, src, t_src, fmt, sign, scale=1.0, stream=None):
    """wire = scale * (psi_up + sign psi_dn) on time slice t_src of the native field src."""
    _check(lib().lq_face_pack(h, _ptr(wire), _ptr(src), int(t_src), fmt, int(sign), float(scale), _stream(stream)),
           "lq_face_pack")


def lq_face_unpack(h, dst, t_dst, wire, fmt, sign, stream=None):
    """Time slice t_dst of the native field dst = the ghost spinor rebuilt from wire for projector sign `sign`."""
    _check(lib().lq_face_unpack(h, _ptr(dst), int(t_dst), _ptr(wire), fmt, int(sign), _stream(stream)),
           "lq_face_unpack")
