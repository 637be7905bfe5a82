/*
 * lqcd.h -- C ABI of the GB300 Wilson / domain-wall Dirac library (liblqcd.so).
 *
 * What is computed.  The paper this library follows (Huth, Meyer, Wettig,
 * "Lattice QCD on a novel vector architecture", Lattice 2019) benchmarks the
 * Wilson Dirac operator (Sec. 3.3, Fig. 4d) built on Grid's stencil/shift
 * (Sec. 3.1) and states no formula for it.  The library implements the
 * textbook operator with these conventions (they are the ones the FP64 CPU
 * oracle in oracle/ is pinned to):
 *
 *   (D psi)(x) = (m + 4) psi(x) - 1/2 (H psi)(x),
 *   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                       + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *   D^dag = gamma_5 D gamma_5  (the same with 1 -/+ gamma swapped),
 *
 * Wilson r = 1, Euclidean chiral basis gamma_k = [[0,-i sigma_k],[i sigma_k,0]]
 * (k = x,y,z), gamma_t = [[0,1],[1,0]], gamma_5 = diag(1,1,-1,-1); a hop that
 * crosses the lattice boundary in direction mu is multiplied by bc[mu].
 * Even-odd: parity(x) = (x0+x1+x2+x3) mod 2, a = m + 4, and the even Schur
 * complement is  Mhat = a - 1/(4a) H_eo H_oe.  Shamir domain wall:
 *   (D_dw psi)(s) = D_W(-M5) psi(s) + psi(s) - P- psi(s+1) - P+ psi(s-1),
 * P+- = (1 +- gamma_5)/2, with P- psi(Ls) := -mf P- psi(0) and
 * P+ psi(-1) := -mf P+ psi(Ls-1); D_dw^dag swaps P+ and P- and uses D_W^dag.
 *
 * Every function returns an int status (LQ_OK = 0, negative on error) and
 * never aborts, exits or throws.  Argument and layout checks run before any
 * launch; a failed check launches nothing.  CUDA errors are returned as
 * LQ_ERR_CUDA.  Apply calls are asynchronous on the given stream; cg_solve
 * returns after the stream has drained, because it fills lq_cg_stats.  A
 * handle is not thread-safe.  All field pointers are DEVICE pointers owned by
 * the caller, 16-byte aligned; outputs must not overlap inputs.
 *
 * ------------------------------------------------------------------ layouts
 * lexi(x) = x0 + L0*(x1 + L1*(x2 + L2*x3)); complex numbers are (re, im).
 *
 * Site-major ("LQ_F64", "LQ_F32"; the documented exchange layout):
 *   gauge   [site][mu 4][row 3][col 3][re,im]        U_mu(x): link x -> x+mu
 *   spinor  [rhs][site][spin 4][colour 3][re,im]     (full field, V sites)
 *   half    [rhs][cb][spin 4][colour 3][re,im]       cb = lexi/2, one parity
 *   5-d     [s][site][spin 4][colour 3][re,im]
 *
 * Native (LQ_NATIVE | precision; the layout the kernels stream): one parity
 * block of Vh = V/2 sites is a set of planes; plane k holds chunk k of every
 * site in cb order (structure of arrays, 16-byte chunks):
 *   LQ_F64:  12 planes x Vh x 16 B, plane k = complex number k
 *            (spin k/3, colour k%3);
 *   LQ_F32:   6 planes x Vh x 16 B, plane k = complex numbers 2k, 2k+1;
 *   LQ_F16 / LQ_BF16: 3 planes x Vh x 16 B (plane k = complex 4k..4k+3,
 *            stored divided by the site norm), then 1 plane x Vh x 4 B of
 *            FP32 site norms (norm = max |real component| of the site).
 * A full native field is [parity 0 block][parity 1 block]; rhs (or s) is the
 * slowest index.  lq_field_bytes() gives every size.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LQ_OK = 0,
    LQ_ERR_ARG = -1,           /* bad argument (null, range, aliasing, unsupported combination) */
    LQ_ERR_LAYOUT = -2,        /* misaligned pointer or unsupported lattice shape */
    LQ_ERR_CUDA = -3,          /* a CUDA runtime call or launch failed */
    LQ_ERR_NOMEM = -4,         /* device allocation failed */
    LQ_ERR_NOT_CONVERGED = -5, /* solver hit maxiter; x holds the best iterate */
    LQ_ERR_BREAKDOWN = -6,     /* solver breakdown (<p,Ap> <= 0, NaN/Inf scalar) */
    LQ_ERR_TIMEOUT = -7,       /* a bounded device-side wait ran out */
    LQ_ERR_NAN = -8            /* NaN or Inf in an input or the residual */
};

/* Precisions; OR with LQ_NATIVE for a native-layout field. */
enum { LQ_F64 = 0, LQ_F32 = 1, LQ_F16 = 2, LQ_BF16 = 3 };
#define LQ_NATIVE 0x10

/* parity argument of the Wilson apply calls */
enum {
    LQ_FULL = -1,       /* in, out: full fields;   out = D in            */
    LQ_EVEN = 0,        /* in: odd half, out: even half; out = D_eo in = -1/2 H_eo in */
    LQ_ODD = 1,         /* in: even half, out: odd half; out = D_oe in = -1/2 H_oe in */
    LQ_SCHUR_EVEN = 2   /* in, out: even halves;    out = Mhat in          */
};

typedef struct {
    int dims[4];     /* L0..L3 (x fastest); each even and >= 2, V/2 < 2^31 */
    int bc[4];       /* +1 periodic, -1 antiperiodic; e.g. {1,1,1,-1} */
    double mass;     /* Wilson bare mass m */
    double r;        /* Wilson r; must be 1 (the kernels use the rank-2 spin projectors) */
    int Ls;          /* domain-wall extent; 0 = no domain-wall operator */
    double M5;       /* domain-wall height */
    double mf;       /* domain-wall quark mass */
    int compress12;  /* 1: links stored as their first two rows, row 3 = conj(row1 x row2) */
    int mobius;      /* 0: Shamir domain wall; 1: Moebius with b5, c5 (FP64/FP32 fields):
                        D_M = (b5 D_W(-M5) + 1) + (c5 D_W(-M5) - 1) S,  S psi(s) = P- psi(s+1) + P+ psi(s-1)
                        (walls -mf); b5 = 1, c5 = 0 is the Shamir operator */
    double b5, c5;   /* Moebius coefficients (read only when mobius = 1) */
} lq_params;

typedef struct lq_handle lq_handle;

/*
 * lq_create: build a handle for one gauge field.
 *   U       device pointer, site-major gauge field in precision U_prec (LQ_F64
 *           or LQ_F32); read during the call only (packed into the handle's
 *           own native copies).  With compress12 = 1 the links must be
 *           SU(3): a link whose |U^dag U - 1| (largest entry) or |det U - 1|
 *           exceeds 1e-6 (FP64 links) or 1e-5 (FP32 links), or holds a NaN,
 *           makes the call fail with LQ_ERR_ARG (no handle is made).
 *   stream  cudaStream_t used for the packing; the call synchronises it.
 * The handle owns its packed links (one copy per precision, made on first
 * use) and its workspace; lq_destroy frees them.
 */
int lq_create(lq_handle **h, const lq_params *p, const void *U, int U_prec, void *stream);
int lq_destroy(lq_handle *h);

/*
 * lq_field_bytes: bytes of a field in format fmt holding nrhs right-hand
 * sides (or Ls slices) of `subset` sites: LQ_FULL (V sites), LQ_EVEN/LQ_ODD
 * (V/2 sites); five_d != 0 multiplies by Ls (the rhs count is then ignored).
 */
int lq_field_bytes(const lq_handle *h, int fmt, int subset, int nrhs, int five_d, size_t *bytes);

/*
 * lq_convert: copy nrhs fields from one format to another (site-major <->
 * native, precision change).  subset as in lq_field_bytes; five_d selects the
 * 5-d layout.  dst and src must not overlap.  Site-major formats are
 * LQ_F64 / LQ_F32; LQ_F16 / LQ_BF16 exist only as native formats.
 * dst and src may be device or managed memory, or pinned host memory mapped
 * into the unified address space (cudaHostAlloc): the conversion kernel then
 * reads or writes host memory over the host link, fusing the transfer with
 * the conversion.  A pointer the device cannot address is LQ_ERR_LAYOUT.
 */
int lq_convert(lq_handle *h, void *dst, int dst_fmt, const void *src, int src_fmt, int subset, int nrhs,
               int five_d, void *stream);

/*
 * dslash_apply / dslash_dag_apply: Wilson operator D (or D^dag) on nrhs
 * fields, as selected by `parity` (LQ_FULL, LQ_EVEN, LQ_ODD, LQ_SCHUR_EVEN).
 * fmt gives layout and arithmetic of in and out: LQ_F64 / LQ_F32 site-major
 * (converted to native and back inside the call, using handle workspace), or
 * LQ_NATIVE | p (streamed directly).  FP64 fields compute in FP64; FP32, FP16
 * and BF16 fields compute in FP32 with links stored in the same precision.
 */
int dslash_apply(lq_handle *h, void *out, const void *in, int fmt, int parity, int nrhs, void *stream);
int dslash_dag_apply(lq_handle *h, void *out, const void *in, int fmt, int parity, int nrhs, void *stream);

/*
 * lq_set_hop_kernel: which kernel computes the Wilson hops of this handle.
 * The paper's kernels are CUDA-core code (Sec. 3.3); the tensor-core variant
 * is this library's own.  LQ_HOP_CUDA_CORES (the default): the CUDA-core hop.
 * LQ_HOP_TENSOR_CORES: a launch of at least 8 right-hand sides (or a
 * domain-wall operator of at least 8 slices, which share each link like
 * right-hand sides) with FP16/BF16 storage and 18-real links, over whole
 * parity blocks, runs its SU(3) x half-spinor products on the tensor cores
 * (one 16x8x8 MMA with FP32 accumulation per site, direction and group of 8
 * right-hand sides or slices); every other launch keeps the CUDA-core hop.  The two
 * agree to the rounding of FP32 sums.  On GB300 the tensor-core variant is
 * the slower of the two (24^3 x 48, 12 right-hand sides, FP16: 1.1 ms against
 * 0.40 ms), so it is not the default.  Takes effect for launches made after
 * the call (a solver captures it when it starts); other kind values are
 * LQ_ERR_ARG.
 */
enum { LQ_HOP_CUDA_CORES = 0, LQ_HOP_TENSOR_CORES = 1 };
int lq_set_hop_kernel(lq_handle *h, int kind);

/*
 * dwf_dslash_apply: domain-wall operator D_dw (dagger != 0: D_dw^dag) on one
 * 5-d field of Ls slices (lq_params.Ls), layout by fmt as above: Shamir, or
 * Moebius when lq_params.mobius = 1 (then FP64/FP32 only, LQ_ERR_ARG else).
 */
int dwf_dslash_apply(lq_handle *h, void *out, const void *in, int fmt, int dagger, void *stream);

/*
 * Even-odd (4-d parity) preconditioned domain wall.  The paper does not treat
 * the domain-wall operator; this is the standard Schur decomposition of D_dw
 * by 4-d parity.  With M5 the part of D_dw that stays on a 4-d site,
 *   (M5 psi)(s) = (5 - M5) psi(s) - P- psi(s+1) - P+ psi(s-1)  (walls -> +mf),
 * and M_eo = -1/2 H_eo, M_oe = -1/2 H_oe (the Wilson hop between parities, on
 * every slice), D_dw psi = eta is solved on the even sites through
 *   Mhat = M5 - M_eo M5^{-1} M_oe,   Mhat psi_e = eta_e - M_eo M5^{-1} eta_o,
 * and psi_o = M5^{-1} (eta_o - M_oe psi_e).
 * Field layouts: a 5-d half field is Ls half fields of the even parity, slice
 * after slice ([s][cb][4][3] site-major, or Ls native blocks); lq_field_bytes
 * and lq_convert handle it as subset LQ_EVEN with nrhs = Ls.  A full 5-d field
 * is the five_d layout above.  fmt: LQ_F64 or LQ_F32, site-major or native
 * (FP16/BF16: LQ_ERR_ARG).  All three are asynchronous on `stream` and
 * reject overlapping buffers (LQ_ERR_ARG); they need lq_params.Ls >= 1.
 * For the Moebius operator (lq_params.mobius = 1), with B = b5 + c5 S, the
 * same three formulas hold with M5 replaced by the site-local part
 *   M5_M = ((4 - M5) b5 + 1) + ((4 - M5) c5 - 1) S
 * and M_eo = -1/2 H_eo B, M_oe = -1/2 H_oe B (B acts before the hop).  A
 * singular M5_M ((4 - M5) b5 + 1 = 0, or 1 + mf g^Ls = 0 with
 * g = (1 - (4 - M5) c5) / ((4 - M5) b5 + 1)) is LQ_ERR_ARG.
 *
 * dwf_schur_apply: out_e = Mhat in_e (dagger != 0: Mhat^dag in_e), 5-d half fields.
 * dwf_eo_prepare: bhat_e = eta_e - M_eo M5^{-1} eta_o from a full 5-d source eta.
 * dwf_eo_reconstruct: the full 5-d solution psi (psi_e = x_e, psi_o as above)
 *   from the even half x_e and the source eta.
 */
int dwf_schur_apply(lq_handle *h, void *out_e, const void *in_e, int fmt, int dagger, void *stream);
int dwf_eo_prepare(lq_handle *h, void *bhat_e, const void *eta, int fmt, void *stream);
int dwf_eo_reconstruct(lq_handle *h, void *psi, const void *x_e, const void *eta, int fmt, void *stream);

/*
 * lq_dot: FP64 complex inner products <a, b> = sum_x conj(a(x)) . b(x) of
 * nrhs pairs of fields (layout and precision fmt, sites as in lq_field_bytes;
 * five_d != 0: one 5-d field of Ls slices).  result: DEVICE pointer to
 * 2 * nrhs doubles, (re, im) per right-hand side, written asynchronously on
 * `stream` (memory the device can address, as for lq_convert: a result or
 * field pointer the device cannot address is LQ_ERR_LAYOUT).  Products are formed in the field's arithmetic precision and
 * summed in FP64 (warp shuffles, one partial per block, fixed-order final
 * sum by the last block), so repeated calls give identical results.  The
 * reduction partials live in handle workspace that grows (cudaMalloc) on
 * first use.  It is the global reduction the CG solvers iterate on (the
 * paper's benchmark, Sec. 3.3, times the operator alone).
 */
int lq_dot(lq_handle *h, double *result, const void *a, const void *b, int fmt, int subset, int nrhs, int five_d,
           void *stream);

/*
 * lq_dot_noalloc: lq_dot for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a service of the library.
 * lq_dot grows handle workspace with cudaMalloc on first use, which some
 * callers cannot allow: code that manages the whole device memory budget
 * through its own pool, latency-critical loops in which cudaMalloc/cudaFree
 * would synchronise the device, and code running while a stream is being
 * captured, where allocation calls fail.  This call runs the same reduction
 * with its scratch in a fixed file-scope device array (about 0.6 MB, held by
 * every GPU that loads the library until the process exits) and calls no
 * allocating routine.  Arguments, result and argument checks are those of
 * lq_dot (a result pointer the device cannot address is LQ_ERR_LAYOUT).
 *   - nrhs (1 for five_d) must be <= LQ_DOT_NOALLOC_MAX_RHS, else LQ_ERR_ARG.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind (the call clears what must start at zero).  Calls whose work
 *     overlaps on the GPU -- concurrent streams, or threads sharing a device
 *     without ordering -- race on the array; order them on one stream.
 */
#define LQ_DOT_NOALLOC_MAX_RHS 32
int lq_dot_noalloc(lq_handle *h, double *result, const void *a, const void *b, int fmt, int subset, int nrhs,
                   int five_d, void *stream);

/*
 * lq_index_faults: the record of the index-checked build.  A library built with
 * -DLQ_INDEX_CHECK (paper_2001_07557_gb300/build.py, build(checked=True), which
 * writes liblqcd_checked.so) compares every neighbour index its hop kernels
 * compute with the parity block before using it; an index out of range is
 * counted, the first one kept, and the access redirected to site 0, so the
 * check cannot fault.  The paper has no counterpart: this is a testing aid that
 * stands in for a device memory checker.
 *   count    receives the indices out of range since the previous call, on the
 *            current device (the call clears the record; it synchronises the device)
 *   first    (may be null) the first such index, -1 if none
 *   checked  (may be null) 1 for the index-checked build, 0 for the normal one,
 *            whose count is always 0
 * Returns LQ_ERR_ARG for a null count, LQ_ERR_CUDA if the record cannot be read.
 */
int lq_index_faults(unsigned long long *count, long long *first, int *checked);

/* ------------------------------------------------------------------- CG */

enum {
    LQ_OP_WILSON_NORMAL = 0,    /* A = D^dag D on full fields           */
    LQ_OP_WILSON_EO_NORMAL = 1, /* A = Mhat^dag Mhat on even half fields */
    LQ_OP_DWF_NORMAL = 2,       /* A = D_dw^dag D_dw on 5-d fields       */
    LQ_OP_DWF_EO_NORMAL = 3     /* A = Mhat^dag Mhat on 5-d even half fields (domain-wall Schur
                                   complement; FP64/FP32, inner precision LQ_F32 only) */
};
enum {
    LQ_CG_PLAIN = 0,   /* CG in the precision of fmt (FP64 or FP32) */
    LQ_CG_MIXED = 1,   /* FP64 defect correction around an inner CG in `inner` precision */
    LQ_CG_BLOCK = 2,   /* block CG over nrhs right-hand sides (inner precision `inner`) */
    LQ_CG_BATCHED = 3  /* nrhs independent CGs sharing each link load */
};

typedef struct {
    int op;            /* LQ_OP_* */
    int mode;          /* LQ_CG_* */
    int fmt;           /* format of x and b (site-major or native) */
    int nrhs;          /* number of right-hand sides (>= 1) */
    double tol;        /* stop when |b - A x| / |b| < tol (per right-hand side) */
    int maxiter;       /* total inner iterations allowed */
    int inner;         /* inner precision for LQ_CG_MIXED / LQ_CG_BLOCK (LQ_F32, LQ_F16, LQ_BF16) */
    double inner_tol;  /* relative reduction asked of each inner solve (0: library default) */
    int x0_is_guess;   /* 1: x holds an initial guess on entry (restart); 0: start from x = 0 */
} lq_cg_params;

typedef struct {
    int iters;                /* total operator applications of A (inner + outer) */
    int outer_iters;          /* defect-correction restarts (0 for plain CG) */
    int status;               /* LQ_OK or an error code for this right-hand side */
    double true_rel_residual; /* |b - A x| / |b| recomputed in FP64 at the end */
    double time_ms;           /* wall time of the solve */
} lq_cg_stats;

/*
 * cg_solve: solve A x = b (A from cp->op) for cp->nrhs right-hand sides.
 * stats must point to cp->nrhs entries.  Returns LQ_OK when every right-hand
 * side reached tol, LQ_ERR_NOT_CONVERGED (x = best iterate) or another error.
 */
int cg_solve(lq_handle *h, void *x, const void *b, const lq_cg_params *cp, lq_cg_stats *stats, void *stream);

/*
 * lq_batch_cg_solve: nlat independent lattices (one handle each), each with
 * cp->nrhs right-hand sides, solved together: every operator and vector step
 * of all lattices is one launch of a persistent kernel walking a work list,
 * and the iteration is captured once in a CUDA graph and replayed.  xs[i],
 * bs[i] belong to hs[i]; stats holds nlat * cp->nrhs entries (lattice-major).
 * The persistent hop's shape -- sites per work item of each lattice (1, 2, 4
 * or 8 tiles of 128) and the resident blocks -- is timed on the batch at its
 * first solve and kept per device model and batch shape.  With the
 * environment variable LQCD_TUNE_CACHE naming a file, the choices are read
 * from and written to it, one line per batch shape:
 *   <key> <blocks> <nlat> <tiles per item of lattice 0> ... (lattice nlat-1)
 */
int lq_batch_cg_solve(lq_handle **hs, int nlat, void **xs, const void **bs, const lq_cg_params *cp,
                      lq_cg_stats *stats, void *stream);

/* ------------------------------------------- time-slab decomposition */

/*
 * Building blocks of a domain decomposition in time: every rank holds a slab
 * of time slices plus one ghost slice on each side (a lattice of its own
 * handle, L3 = slab + 2), fills the ghosts from its neighbours' edge slices
 * before each hop, and keeps the output of its own slices.  The paper's MPI
 * shift (Sec. 3.2) is unfinished; these calls carry the same exchange between
 * handles on one device.
 *
 * dslash_apply_slices: the full-lattice Wilson operator D (dagger != 0: D^dag)
 *   with output on the time slices t0 <= t < t1 only; other sites of out are
 *   not written.  in and out are full native fields (fmt = LQ_NATIVE | prec;
 *   site-major formats give LQ_ERR_LAYOUT).  0 <= t0 < t1 <= L3.  Computing
 *   the slab's interior slices while the ghosts are copied, then its two edge
 *   slices, overlaps the exchange with the hop.
 *
 * lq_face_copy: time slice t_src of src (a full native field of hs's lattice)
 *   times scale, into time slice t_dst of dst (a full native field of hd's
 *   lattice).  hd and hs must have the same L0, L1, L2 (LQ_ERR_ARG).  scale is
 *   +1, or -1 where the copy crosses the global antiperiodic time boundary
 *   (FP16/BF16 fields carry it in their site norms).  If t_dst - t_src is odd
 *   the local parities of the slice's sites differ between the two lattices and
 *   the parity blocks are swapped.  dst and src may be one field if the slices
 *   differ.  Asynchronous on `stream`.
 */
int dslash_apply_slices(lq_handle *h, void *out, const void *in, int fmt, int t0, int t1, int dagger, void *stream);
int lq_face_copy(lq_handle *hd, void *dst, int t_dst, lq_handle *hs, const void *src, int t_src, int fmt, double scale,
                 void *stream);

/*
 * Spin-projected faces: the exchange of lq_face_copy at half the bytes.  A hop
 * reads a ghost slice only through the time-direction projector, (1 + S gamma_t)
 * with S = +1 for the ghost below the slab and S = -1 for the ghost above it
 * (D^dag: the opposite signs).  In the chiral basis gamma_t = [[0, 1], [1, 0]],
 * (1 + S gamma_t) psi = [h; S h] with h = psi_up + S psi_dn, 2 spins x 3 colours,
 * so only h has to travel (the halo exchange of Sec. 3.2 would send it between
 * ranks; here a cudaMemcpyAsync between two wire buffers stands in for it).
 *
 * Wire layout (the only format on the wire; both sides are native fields of
 * precision fmt & 0xF): two blocks, one per spatial parity (x0 + x1 + x2) mod 2,
 * of V3/2 sites (V3 = L0 L1 L2) in the slice's run order.  Per block: FP64
 * 6 planes of 16 B, FP32 3 planes of 16 B, FP16/BF16 3 planes of 8 B followed
 * by one FP32 norm per site.  Because the wire is indexed by spatial parity,
 * sender and receiver slices may differ by any distance.
 *
 * lq_face_wire_bytes: bytes of one wire buffer for h's slices (L0 L1 L2 / 2
 *   sites per block) in format fmt.
 * lq_face_pack: wire = scale * h of time slice t_src of src (a full native
 *   field of h's lattice) for projector sign S = sign (+1 or -1).  scale is
 *   +1, or -1 across the global antiperiodic time boundary.
 * lq_face_unpack: time slice t_dst of dst (a full native field of h's
 *   lattice) = the ghost spinor chi = [h/2; S h/2] (FP16/BF16: [h; S h] with
 *   the norm halved), whose projection chi_up + S chi_dn is h exactly: a hop
 *   that reads the ghost through (1 + S gamma_t) then reproduces the
 *   single-domain result bit for bit.  The other spin components of the
 *   ghost are not those of psi; only a hop through the same projector may
 *   read it.
 * Both: the field must be native (LQ_ERR_LAYOUT otherwise) and 16-byte
 * aligned, as must the wire (LQ_ERR_LAYOUT); sign not +-1, t out of range or
 * an overlap of field and wire is LQ_ERR_ARG.  Asynchronous on `stream`.
 */
int lq_face_wire_bytes(const lq_handle *h, int fmt, size_t *bytes);
int lq_face_pack(lq_handle *h, void *wire, const void *src, int t_src, int fmt, int sign, double scale, void *stream);
int lq_face_unpack(lq_handle *h, void *dst, int t_dst, const void *wire, int fmt, int sign, void *stream);

/* ---------------------------------------------------- SU(3) x SU(3) */

/*
 * lq_su3_mul: the lattice-wide colour-matrix product of the paper's SU(3)
 * matrix-matrix benchmark (Sec. 3.3, Fig. 4a-c):  C[x] = A[x] B[x],
 * C_ij = sum_k A_ik B_kj, for x = 0 .. n-1.
 *   - A, B, C: device pointers to n 3x3 complex matrices stored
 *     [x][row][col] as interleaved {re, im} pairs (the paper's array of
 *     two-element structures), FP64 (fmt = LQ_F64, 144 bytes per matrix) or
 *     FP32 (fmt = LQ_F32, 72 bytes).  Each must be 16-byte aligned
 *     (LQ_ERR_LAYOUT otherwise).  The caller owns all three.
 *   - C may be the same pointer as A or as B (the product is formed in place
 *     tile by tile); any other overlap is LQ_ERR_ARG.
 *   - n = 0 is a no-op; n < 0 or a null pointer with n > 0 is LQ_ERR_ARG.
 *   - Asynchronous on `stream`.  No handle is needed and nothing is allocated.
 * Tiles of A and B move to shared memory by bulk asynchronous copies that
 * complete on shared-memory barriers, and tiles of C leave by bulk stores.
 * Every wait on a barrier is bounded (about a second); a wait that runs out
 * leaves its tile of C, and the later tiles of its block, unwritten and is
 * counted.  The call is asynchronous, so it cannot report that itself: its
 * status covers the argument checks and the launch.  lq_wait_timeouts
 * (which synchronises) reports it as LQ_ERR_TIMEOUT.
 */
int lq_su3_mul(void *C, const void *A, const void *B, long n, int fmt, void *stream);

/*
 * lq_wait_timeouts: the number of device-side barrier waits that ran out
 * since the last call (on the current device), then reset to zero.
 * Synchronises the device.  Returns LQ_ERR_TIMEOUT when the count is not
 * zero (it is still written): some results of the kernels that wait on
 * barriers (lq_su3_mul) were not written.  LQ_OK otherwise.
 */
int lq_wait_timeouts(unsigned *count);

/*
 * lq_test_stalled_wait: exercises the timeout path of the barrier waits.  It
 * runs the SU(3) product kernel on one tile of zero matrices (in its own
 * scratch) with the stage barrier armed for 16 more bytes than the copies
 * bring, so that the phase never completes: the bounded wait gives up after
 * about a second, the kernel returns, and the count read by lq_wait_timeouts
 * grows by one.  No fault and no hang; the device stays usable.  Synchronises
 * the device.  For tests of the failure path only.
 */
int lq_test_stalled_wait(void);

/* Human-readable text for a status code (static storage). */
const char *lq_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
