// cg.cu -- conjugate gradient on the normal equations A x = b,
// A = K^dag K for K = D (full lattice), Mhat (even-odd Schur complement) or
// D_dw (domain wall), for nrhs right-hand sides at once.
//
//  * plain CG (Hestenes-Stiefel) in FP64 or FP32;
//  * mixed precision: an FP64 defect-correction loop (true residual
//    r = b - A x in FP64 on the GPU) around an inner CG whose search
//    directions and operator live in FP32, FP16 or BF16 storage (FP32
//    arithmetic) and whose iterate and residual are FP32;
//  * every right-hand side keeps its own device-resident scalars; the
//    reductions are fused into the vector updates and finish on the device,
//    the iteration is captured once into a CUDA graph and replayed, and the
//    host polls the scalars once per graph replay.
// The paper (Sec. 3.3) benchmarks the Wilson operator only; the solver
// around it follows the textbook CG.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "blas.h"
#include "blockcg.h"
#include "handle.h"
#include "trace.h"

namespace lq {

namespace {

constexpr int kItersPerGraph = 8;

struct OpGeom {
    int op;
    int nblk;   // parity blocks per right-hand side
    int nrhs;
    size_t stride(const lq_handle* h, int prec) const {
        return (size_t)nblk * spinor_site_bytes(prec) * (size_t)h->g.Vh;
    }
    size_t bytes(const lq_handle* h, int prec) const { return stride(h, prec) * nrhs; }
    // the odd-parity scratch of one operator application: nrhs blocks, or Ls for the domain-wall Schur complement
    size_t tmp_bytes(const lq_handle* h, int prec) const {
        return (size_t)spinor_site_bytes(prec) * h->g.Vh * (op == LQ_OP_DWF_EO_NORMAL ? h->p.Ls : nrhs);
    }
    VecRef ref(const lq_handle* h, void* p, int prec) const { return VecRef{static_cast<char*>(p), prec, stride(h, prec)}; }
};

// out = K^dag K in;  t: intermediate of in's size, tmp: odd half (even-odd only).
// With c given, the launch that writes t = K in also sums |t|^2 = <in, K^dag K in>
// per right-hand side and sets the CG step length alpha on the device.
struct Ctl;
int apply_normal(lq_handle* h, const OpGeom& og, int prec, char* out, const char* in, char* t, char* tmp,
                 cudaStream_t st, const Ctl* c = nullptr);

// Solver scratch: scalars, norms, reduction partials, tickets (one workspace slot)
struct Ctl {
    CgScalars* st;
    double* red;  // 2 * nrhs doubles
    Scratch sc;
    CgScalars* host;
    double* hop_partial;  // fused |K p|^2 partials of the hop launches
    unsigned* hop_tickets;
};

int ensure_pinned(lq_handle* h, size_t hb) {
    if (h->pinned_bytes < hb) {
        if (h->pinned) cudaFreeHost(h->pinned);
        h->pinned = nullptr;
        h->pinned_bytes = 0;
        if (cudaMallocHost(&h->pinned, hb) != cudaSuccess) {
            cudaGetLastError();
            return LQ_ERR_NOMEM;
        }
        h->pinned_bytes = hb;
    }
    return LQ_OK;
}

int make_ctl(lq_handle* h, const OpGeom& og, Ctl* c, cudaStream_t s) {
    const size_t npart = reduce_scratch_doubles(h->g.Vh, og.nblk, og.nrhs);
    const size_t nhop = hop_red_warps(h->g.Vh, 2, std::max(h->p.Ls, 1)) * (size_t)og.nrhs;
    const size_t nb = sizeof(CgScalars) * og.nrhs + sizeof(double) * (2 * og.nrhs + npart + nhop) +
                      2 * sizeof(unsigned) * og.nrhs + 256;
    void* p;
    int rc = ensure_ws(h, WS_CTL, nb, &p);
    if (rc) return rc;
    char* q = static_cast<char*>(p);
    c->st = reinterpret_cast<CgScalars*>(q);
    q += sizeof(CgScalars) * og.nrhs;
    c->red = reinterpret_cast<double*>(q);
    q += sizeof(double) * 2 * og.nrhs;
    c->sc.partial = reinterpret_cast<double*>(q);
    q += sizeof(double) * npart;
    c->hop_partial = reinterpret_cast<double*>(q);
    q += sizeof(double) * nhop;
    c->sc.tickets = reinterpret_cast<unsigned*>(q);
    c->hop_tickets = c->sc.tickets + og.nrhs;
    if (cudaMemsetAsync(c->sc.tickets, 0, 2 * sizeof(unsigned) * og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
    const size_t hb = sizeof(CgScalars) * og.nrhs + sizeof(double) * 2 * og.nrhs;
    if ((rc = ensure_pinned(h, hb))) return rc;
    c->host = static_cast<CgScalars*>(h->pinned);
    return LQ_OK;
}

// t = K in, the first half of the normal operator (with the fused |K in|^2 when c is given)
int apply_k(lq_handle* h, const OpGeom& og, int prec, char* t, const char* in, char* tmp, cudaStream_t st,
            const Ctl* c = nullptr) {
    int rc;
    if (c) {
        h->red_partial = c->hop_partial;
        h->red_ticket = c->hop_tickets;
        h->red_st = c->st;
    }
    switch (og.op) {
    case LQ_OP_WILSON_NORMAL: rc = native_wilson_full(h, prec, t, in, og.nrhs, false, st); break;
    case LQ_OP_WILSON_EO_NORMAL: rc = native_wilson_schur(h, prec, t, in, tmp, og.nrhs, false, st); break;
    case LQ_OP_DWF_NORMAL: rc = native_dwf(h, prec, t, in, false, st); break;
    case LQ_OP_DWF_EO_NORMAL: rc = native_dwf_schur(h, prec, t, in, tmp, false, st); break;
    default: rc = LQ_ERR_ARG;
    }
    h->red_partial = nullptr;
    h->red_ticket = nullptr;
    h->red_st = nullptr;
    return rc;
}

// out = K^dag t, the second half
int apply_kdag(lq_handle* h, const OpGeom& og, int prec, char* out, const char* t, char* tmp, cudaStream_t st) {
    switch (og.op) {
    case LQ_OP_WILSON_NORMAL: return native_wilson_full(h, prec, out, t, og.nrhs, true, st);
    case LQ_OP_WILSON_EO_NORMAL: return native_wilson_schur(h, prec, out, t, tmp, og.nrhs, true, st);
    case LQ_OP_DWF_EO_NORMAL: return native_dwf_schur(h, prec, out, t, tmp, true, st);
    default: return native_dwf(h, prec, out, t, true, st);
    }
}

int apply_normal(lq_handle* h, const OpGeom& og, int prec, char* out, const char* in, char* t, char* tmp,
                 cudaStream_t st, const Ctl* c) {
    const int rc = apply_k(h, og, prec, t, in, tmp, st, c);
    return rc ? rc : apply_kdag(h, og, prec, out, t, tmp, st);
}

// warp partials per group written by the fused-norm launch of apply_normal
int hop_warps(const lq_handle* h, const OpGeom& og) {
    switch (og.op) {
    case LQ_OP_WILSON_NORMAL: return (int)hop_red_warps(h->g.Vh, 2, 1);
    case LQ_OP_WILSON_EO_NORMAL: return (int)hop_red_warps(h->g.Vh, 1, 1);
    case LQ_OP_DWF_EO_NORMAL: return (int)hop_red_warps(h->g.Vh, 1, h->p.Ls);
    default: return (int)hop_red_warps(h->g.Vh, 2, h->p.Ls);
    }
}

double* host_red(lq_handle* h, const OpGeom& og) {
    return reinterpret_cast<double*>(static_cast<char*>(h->pinned) + sizeof(CgScalars) * og.nrhs);
}

// norms |v|^2 of every rhs into host memory
int norms_to_host(lq_handle* h, const OpGeom& og, const Ctl& c, const VecRef& v, double* out, cudaStream_t s) {
    if (launch_dot(v, v, h->g.Vh, og.nblk, og.nrhs, c.sc, nullptr, c.red, FIN_STORE, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    double* hr = host_red(h, og);
    if (cudaMemcpyAsync(hr, c.red, sizeof(double) * og.nrhs, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LQ_ERR_CUDA;
    for (int k = 0; k < og.nrhs; ++k) out[k] = hr[k];
    return LQ_OK;
}

struct CgVecs {
    VecRef r, p, q, t, tmp;  // r in the iterate precision; p, q, t, tmp in the operator precision
};

int cg_vectors(lq_handle* h, const OpGeom& og, int px, int pp, int slot0, CgVecs* v) {
    void* ptr[5];
    const size_t sz[5] = {og.bytes(h, px), og.bytes(h, pp), og.bytes(h, pp), og.bytes(h, pp), og.tmp_bytes(h, pp)};
    for (int k = 0; k < 5; ++k) {
        int rc = ensure_ws(h, slot0 + k, sz[k], &ptr[k]);
        if (rc) return rc;
    }
    v->r = og.ref(h, ptr[0], px);
    v->p = og.ref(h, ptr[1], pp);
    v->q = og.ref(h, ptr[2], pp);
    v->t = og.ref(h, ptr[3], pp);
    v->tmp = VecRef{static_cast<char*>(ptr[4]), pp, (size_t)spinor_site_bytes(pp) * h->g.Vh};
    return LQ_OK;
}

// CG on A e = rhs.  e, rhs, r in precision px; p, q, t in pp.  Starts from
// e = 0.  Stops per rhs at |r| <= tol |rhs| or after maxiter iterations.
// On return c.host holds the final scalars of every rhs.
int run_cg(lq_handle* h, const OpGeom& og, const Ctl& c, int pp, const VecRef& e, const VecRef& rhs, double tol,
           int maxiter, int slot0, cudaStream_t s) {
    lq::TraceRange trace_("lqcd/cg/inner");
    const int px = e.prec;
    // with FP16/BF16 search directions the residual is kept in the same 16-bit storage
    // (FP32 arithmetic, per-site norms): the update and xpay then move 19% fewer bytes
    const int pr = (px == LQ_F32 && (pp == LQ_F16 || pp == LQ_BF16)) ? pp : px;
    CgVecs v;
    int rc = cg_vectors(h, og, pr, pp, slot0, &v);
    if (rc) return rc;
    const char* L;
    size_t lb;
    if ((rc = get_links(h, pp, &L, &lb, s))) return rc;  // pack before any capture
    if (og.op == LQ_OP_DWF_NORMAL && h->p.mobius) {       // the Moebius operator's 5-d temporaries, likewise
        void* w;
        const size_t f5 = og.bytes(h, pp);
        if ((rc = ensure_ws(h, WS_MOB, f5, &w)) || (rc = ensure_ws(h, WS_MOB + 1, f5, &w))) return rc;
    }
    if (og.op == LQ_OP_DWF_EO_NORMAL && h->p.mobius) {    // and the even-odd Moebius operator's one half field
        void* w;
        if ((rc = ensure_ws(h, WS_MOB, og.bytes(h, pp), &w))) return rc;
    }
    const int Vh = h->g.Vh;
    if (cudaMemsetAsync(e.ptr, 0, og.bytes(h, px), s) != cudaSuccess) return LQ_ERR_CUDA;
    if (pr == px ? cudaMemcpyAsync(v.r.ptr, rhs.ptr, og.bytes(h, px), cudaMemcpyDeviceToDevice, s) != cudaSuccess
                 : launch_axpby(v.r, rhs, 1.0, 0.0, Vh, og.nblk, og.nrhs, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    if (launch_axpby(v.p, v.r, 1.0, 0.0, Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
    if (launch_dot(rhs, rhs, Vh, og.nblk, og.nrhs, c.sc, nullptr, c.red, FIN_STORE, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    if (launch_cg_init(c.st, c.red, c.red, tol, maxiter, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;

    // one graph = kItersPerGraph iterations; finished right-hand sides skip every launch
    h->skip = &c.st[0].done;
    h->skip_stride = (int)(sizeof(CgScalars) / sizeof(int));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    rc = LQ_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = LQ_ERR_CUDA;
    for (int k = 0; k < kItersPerGraph && rc == LQ_OK; ++k) {
        // q = K^dag K p, with <p, q> = |K p|^2 and alpha fused into the launch that writes K p
        rc = apply_normal(h, og, pp, v.q.ptr, v.p.ptr, v.t.ptr, v.tmp.ptr, s, &c);
        if (rc) break;
        if (launch_hop_norm_finalize(c.hop_partial, hop_warps(h, og), og.op == LQ_OP_DWF_NORMAL ? 1 : og.nrhs, c.st,
                                     c.sc, Vh, og.nblk, s) != cudaSuccess) {
            rc = LQ_ERR_CUDA;
            break;
        }
        if (launch_cg_update(e, v.p, v.r, v.q, Vh, og.nblk, og.nrhs, c.sc, c.st, s) != cudaSuccess ||
            launch_cg_xpay(v.p, v.r, Vh, og.nblk, og.nrhs, c.st, s) != cudaSuccess)
            rc = LQ_ERR_CUDA;
    }
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    h->skip = nullptr;
    if (rc == LQ_OK && ce != cudaSuccess) rc = LQ_ERR_CUDA;
    const int key[4] = {og.op, pp, pr, og.nrhs};
    if (rc == LQ_OK) rc = cached_graph_exec(h, key, graph, &exec);
    const int max_launches = maxiter / kItersPerGraph + 2;
    for (int it = 0; rc == LQ_OK && it < max_launches; ++it) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess ||
            cudaMemcpyAsync(c.host, c.st, sizeof(CgScalars) * og.nrhs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = LQ_ERR_CUDA;
            break;
        }
        bool all = true;
        for (int k = 0; k < og.nrhs; ++k) all = all && c.host[k].done;
        if (all) break;
    }
    if (graph) cudaGraphDestroy(graph);  // the executable graph stays with the handle
    cudaGetLastError();
    return rc;
}

// |b - A x| / |b| per rhs in FP64 (x64, b64 native FP64)
int true_residual(lq_handle* h, const OpGeom& og, const Ctl& c, const VecRef& x64, const VecRef& b64, int slot0,
                  double* rel, cudaStream_t s) {
    lq::TraceRange trace_("lqcd/cg/true_residual");
    CgVecs v;
    int rc = cg_vectors(h, og, LQ_F64, LQ_F64, slot0, &v);
    if (rc) return rc;
    if ((rc = apply_normal(h, og, LQ_F64, v.q.ptr, x64.ptr, v.t.ptr, v.tmp.ptr, s))) return rc;
    if (launch_axpby(v.r, b64, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
    if (launch_axpby(v.r, v.q, -1.0, 1.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
    std::vector<double> rr(og.nrhs), bb(og.nrhs);
    if ((rc = norms_to_host(h, og, c, v.r, rr.data(), s))) return rc;
    if ((rc = norms_to_host(h, og, c, b64, bb.data(), s))) return rc;
    for (int k = 0; k < og.nrhs; ++k) rel[k] = bb[k] > 0 ? std::sqrt(rr[k] / bb[k]) : std::sqrt(rr[k]);
    return LQ_OK;
}

// x += e, with A e = b - A x solved from e = 0 by run_cg for the right-hand
// sides in `want` whose true residual |b - A x| is not below tol |b| (the
// others get e = 0), to the reduction that meets margin * tol relative to |b|.
// x, b native in precision wp (CG precision wp).  Adds the iterations to
// iters[k] and takes the CG's status into status[k] for those right-hand
// sides.  Scratch: WS_TMP, WS_CG0 .. WS_CG0 + 4, WS_CG0 + 10.
int correction_cg(lq_handle* h, const OpGeom& og, const Ctl& c, int wp, const VecRef& X, const VecRef& B,
                  double tol, double margin, const std::vector<char>& want, int maxiter, cudaStream_t s, int* iters,
                  int* status) {
    void *x0, *r0;
    int rc;
    if ((rc = ensure_ws(h, WS_TMP, og.bytes(h, wp), &x0)) || (rc = ensure_ws(h, WS_CG0 + 10, og.bytes(h, wp), &r0)))
        return rc;
    const VecRef X0 = og.ref(h, x0, wp), R0 = og.ref(h, r0, wp);
    if (cudaMemcpyAsync(x0, X.ptr, og.bytes(h, wp), cudaMemcpyDeviceToDevice, s) != cudaSuccess) return LQ_ERR_CUDA;
    CgVecs v;
    if ((rc = cg_vectors(h, og, wp, wp, WS_CG0, &v))) return rc;
    if ((rc = apply_normal(h, og, wp, v.q.ptr, X0.ptr, v.t.ptr, v.tmp.ptr, s))) return rc;
    if (launch_axpby(R0, B, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess ||
        launch_axpby(R0, v.q, -1.0, 1.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    std::vector<double> bb(og.nrhs), r0n(og.nrhs);
    if ((rc = norms_to_host(h, og, c, B, bb.data(), s)) || (rc = norms_to_host(h, og, c, R0, r0n.data(), s)))
        return rc;
    // the reduction of |r0| that meets the target relative to |b|; a right-hand side that
    // needs none keeps e = 0
    double t = 1.0;
    bool any = false;
    std::vector<char> solve(og.nrhs, 0);
    for (int k = 0; k < og.nrhs; ++k) {
        if (want[k] && r0n[k] > tol * tol * bb[k]) {
            any = true;
            solve[k] = 1;
            t = std::min(t, margin * tol * std::sqrt(bb[k] / r0n[k]));
        } else if (cudaMemsetAsync(R0.ptr + k * R0.rhs_stride, 0, R0.rhs_stride, s) != cudaSuccess) {
            return LQ_ERR_CUDA;
        }
    }
    if (!any) return LQ_OK;
    if ((rc = run_cg(h, og, c, wp, X, R0, t, maxiter, WS_CG0, s))) return rc;
    if (launch_axpby(X, X0, 1.0, 1.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
    for (int k = 0; k < og.nrhs; ++k) {
        if (!solve[k]) continue;
        iters[k] += c.host[k].iter;
        status[k] = c.host[k].status;
    }
    return LQ_OK;
}

struct BlockCtx {
    lq_handle* h;
    const OpGeom* og;
    char* t;
    char* tmp;
    cudaStream_t s;
};

// stage 0: t = K in; stage 1: out = K^dag t
int block_apply(void* ctx, char* out, const char* in, int stage) {
    BlockCtx* c = static_cast<BlockCtx*>(ctx);
    return stage == 0 ? apply_k(c->h, *c->og, LQ_F32, c->t, in, c->tmp, c->s)
                      : apply_kdag(c->h, *c->og, LQ_F32, out, c->t, c->tmp, c->s);
}

// FP32 residuals of the middle level are accurate to roughly this relative size.
constexpr double kMiddleTol = 1e-5;

// A e = rhs to relative tolerance `target` with an FP32 defect correction:
// e, rhs FP32; each pass solves A d = r with the low-precision inner CG to
// max(itol, what is still needed), adds d to e, and recomputes r = rhs - A e
// with FP32 hops.  iters[k] accumulates operator applications; breakdown[k]
// is set when an inner CG broke down at its first step.
int solve_fp32_middle(lq_handle* h, const OpGeom& og, const Ctl& c, int ip, const VecRef& e, const VecRef& rhs,
                      double target, double itol, int maxiter, cudaStream_t s, int* iters, int* most_out,
                      char* breakdown) {
    lq::TraceRange trace_("lqcd/cg/fp32_middle");
    const int Vh = h->g.Vh, nr = og.nrhs;
    void *rp, *dp, *qp, *tp, *tmpp;
    int rc;
    if ((rc = ensure_ws(h, 20, og.bytes(h, LQ_F32), &rp)) || (rc = ensure_ws(h, 21, og.bytes(h, LQ_F32), &dp)) ||
        (rc = ensure_ws(h, 22, og.bytes(h, LQ_F32), &qp)) || (rc = ensure_ws(h, 23, og.bytes(h, LQ_F32), &tp)) ||
        (rc = ensure_ws(h, 16, og.tmp_bytes(h, LQ_F32), &tmpp)))
        return rc;
    const VecRef R = og.ref(h, rp, LQ_F32), Dv = og.ref(h, dp, LQ_F32), Q = og.ref(h, qp, LQ_F32);
    std::vector<double> bb(nr), rr(nr);
    if ((rc = norms_to_host(h, og, c, rhs, bb.data(), s))) return rc;
    if (cudaMemsetAsync(e.ptr, 0, og.bytes(h, LQ_F32), s) != cudaSuccess ||
        cudaMemcpyAsync(R.ptr, rhs.ptr, og.bytes(h, LQ_F32), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    int used = 0, most = 0;
    std::vector<double> rel(nr, 1.0);
    for (int pass = 0; pass < 8 && used < maxiter; ++pass) {
        double reach = 0.5;
        for (int k = 0; k < nr; ++k)
            if (rel[k] > target && rel[k] > 0) reach = std::min(reach, 0.5 * target / rel[k]);
        if ((rc = run_cg(h, og, c, ip, Dv, R, std::max(itol, reach), maxiter - used, WS_CG0, s))) return rc;
        int m = 0;
        for (int k = 0; k < nr; ++k) {
            iters[k] += c.host[k].iter;
            m = std::max(m, c.host[k].iter);
            // <p, A p> not positive at the first step, with p = r != 0: A is singular on r
            if (c.host[k].status == LQ_ERR_BREAKDOWN && c.host[k].iter == 0) breakdown[k] = 1;
        }
        used += std::max(m, 1);
        most += m;
        if (launch_axpby(e, Dv, 1.0, 1.0, Vh, og.nblk, nr, s) != cudaSuccess) return LQ_ERR_CUDA;
        // r = rhs - A e in FP32
        if ((rc = apply_normal(h, og, LQ_F32, Q.ptr, e.ptr, static_cast<char*>(tp), static_cast<char*>(tmpp), s)))
            return rc;
        if (launch_axpby(R, rhs, 1.0, 0.0, Vh, og.nblk, nr, s) != cudaSuccess ||
            launch_axpby(R, Q, -1.0, 1.0, Vh, og.nblk, nr, s) != cudaSuccess)
            return LQ_ERR_CUDA;
        if ((rc = norms_to_host(h, og, c, R, rr.data(), s))) return rc;
        bool done = true;
        for (int k = 0; k < nr; ++k) {
            iters[k] += 1;
            rel[k] = bb[k] > 0 ? std::sqrt(rr[k] / bb[k]) : 0.0;
            done = done && (rel[k] <= target || !std::isfinite(rel[k]));
        }
        if (done) break;
    }
    *most_out = most;
    return LQ_OK;
}

double default_inner_tol(int prec) {
    switch (prec) {
    case LQ_F32: return 1e-6;
    case LQ_F16: return 1e-3;
    default: return 3e-2;
    }
}

}  // namespace

}  // namespace lq

using namespace lq;

extern "C" int cg_solve(lq_handle* h, void* x, const void* b, const lq_cg_params* cp, lq_cg_stats* stats,
                        void* stream) {
    lq::TraceRange trace_("lqcd/cg_solve");
    if (!h || !x || !b || !cp || !stats) return LQ_ERR_ARG;
    if (!valid_fmt(cp->fmt) || cp->nrhs < 1 || cp->maxiter < 1 || !(cp->tol > 0)) return LQ_ERR_ARG;
    if (!aligned16(x) || !aligned16(b)) return LQ_ERR_LAYOUT;
    const int fprec = cp->fmt & 0xF;
    const bool native = (cp->fmt & LQ_NATIVE) != 0;
    if (fprec > LQ_F32) return LQ_ERR_ARG;  // x and b are FP64 or FP32 fields
    OpGeom og;
    og.op = cp->op;
    og.nrhs = cp->nrhs;
    int subset;
    switch (cp->op) {
    case LQ_OP_WILSON_NORMAL: og.nblk = 2; subset = LQ_FULL; break;
    case LQ_OP_WILSON_EO_NORMAL: og.nblk = 1; subset = LQ_EVEN; break;
    case LQ_OP_DWF_NORMAL:
        if (h->p.Ls < 1 || cp->nrhs != 1) return LQ_ERR_ARG;
        // the Moebius operator's 5th-dimension kernels exist for FP64/FP32 only
        if (h->p.mobius && cp->mode != LQ_CG_PLAIN && cp->inner != LQ_F32) return LQ_ERR_ARG;
        og.nblk = 2 * h->p.Ls;
        subset = LQ_FULL;
        break;
    case LQ_OP_DWF_EO_NORMAL:
        // Ls even half fields; the site-local inverse M5^{-1} exists for FP64/FP32 fields
        if (h->p.Ls < 1 || cp->nrhs != 1 || (fprec != LQ_F64 && fprec != LQ_F32)) return LQ_ERR_ARG;
        if (cp->mode != LQ_CG_PLAIN && cp->inner != LQ_F32) return LQ_ERR_ARG;
        og.nblk = h->p.Ls;
        subset = LQ_EVEN;
        break;
    default: return LQ_ERR_ARG;
    }
    const int mode = cp->mode == LQ_CG_BATCHED ? LQ_CG_MIXED : cp->mode;
    if (mode != LQ_CG_PLAIN && mode != LQ_CG_MIXED && mode != LQ_CG_BLOCK) return LQ_ERR_ARG;
    if (mode == LQ_CG_MIXED && (cp->inner < LQ_F32 || cp->inner > LQ_BF16)) return LQ_ERR_ARG;
    const bool dwf = cp->op == LQ_OP_DWF_NORMAL || cp->op == LQ_OP_DWF_EO_NORMAL;
    if (mode == LQ_CG_BLOCK && (cp->nrhs > kMaxBlockRhs || dwf)) return LQ_ERR_ARG;
    const int nf = dwf ? h->p.Ls : cp->nrhs;  // fields in the user's buffers
    const size_t ub = field_bytes(h, cp->fmt, subset, nf);
    if (overlap(x, ub, b, ub)) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(user) != cudaSuccess) return LQ_ERR_CUDA;
    if (!h->solver_stream && cudaStreamCreateWithFlags(&h->solver_stream, cudaStreamNonBlocking) != cudaSuccess)
        return LQ_ERR_CUDA;
    cudaStream_t s = h->solver_stream;
    const bool full = subset == LQ_FULL;
    const int parity = full ? 0 : LQ_EVEN;
    const int wp = mode == LQ_CG_PLAIN ? fprec : LQ_F64;  // precision of x and b inside the solver

    int rc;
    Ctl c;
    if ((rc = make_ctl(h, og, &c, s))) return rc;
    void *xw, *bw;
    if ((rc = ensure_ws(h, WS_IN, og.bytes(h, wp), &bw)) || (rc = ensure_ws(h, WS_OUT, og.bytes(h, wp), &xw)))
        return rc;
    // user fields -> native working precision
    auto to_native = [&](void* dst, const void* src) -> cudaError_t {
        if (native) return launch_native_convert(wp, dst, fprec, src, h->g.Vh, og.nblk * og.nrhs, s);
        return launch_spinor_to_native(wp, dst, fprec, src, h->g, full, parity, nf, s);
    };
    if (to_native(bw, b) != cudaSuccess) return LQ_ERR_CUDA;
    VecRef X = og.ref(h, xw, wp), B = og.ref(h, bw, wp);
    std::vector<int> iters(og.nrhs, 0), status(og.nrhs, LQ_OK), outer(og.nrhs, 0);
    std::vector<double> rel(og.nrhs, 0.0);

    if (mode == LQ_CG_PLAIN) {
        // FP64: the recursive residual is taken to half of tol, so that the true residual, which
        // drifts from it by rounding, lands below tol (a restart below covers the rare miss; a
        // restart loses the Krylov space and costs far more than the few extra iterations)
        const double first = wp == LQ_F64 ? 0.5 : 1.0;
        if (cp->x0_is_guess) {
            // restart from a guess: solve A e = b - A x0, then x = x0 + e
            if (to_native(xw, x) != cudaSuccess) return LQ_ERR_CUDA;
            const std::vector<char> all(og.nrhs, 1);
            if ((rc = correction_cg(h, og, c, wp, X, B, cp->tol, first, all, cp->maxiter, s, iters.data(),
                                    status.data())))
                return rc;
        } else {
            if ((rc = run_cg(h, og, c, wp, X, B, first * cp->tol, cp->maxiter, WS_CG0, s))) return rc;
            for (int k = 0; k < og.nrhs; ++k) {
                iters[k] = c.host[k].iter;
                status[k] = c.host[k].status;
            }
        }
        // true residual in FP64
        void *x64 = nullptr, *b64 = nullptr;
        if (wp != LQ_F64 && ((rc = ensure_ws(h, WS_CG0 + 11, og.bytes(h, LQ_F64), &x64)) ||
                             (rc = ensure_ws(h, WS_CG0 + 12, og.bytes(h, LQ_F64), &b64))))
            return rc;
        auto residual = [&]() -> int {
            if (wp == LQ_F64) return true_residual(h, og, c, X, B, WS_CG0 + 5, rel.data(), s);
            VecRef X64 = og.ref(h, x64, LQ_F64), B64 = og.ref(h, b64, LQ_F64);
            if (launch_axpby(X64, X, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess ||
                launch_axpby(B64, B, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess)
                return LQ_ERR_CUDA;
            return true_residual(h, og, c, X64, B64, WS_CG0 + 5, rel.data(), s);
        };
        if ((rc = residual())) return rc;
        if (wp == LQ_F64) {
            // reliable stop: CG stops on its recursive residual, which drifts from the true one
            // by rounding; a right-hand side whose FP64 true residual is not yet below tol
            // restarts from its iterate (up to three times, within maxiter)
            for (int pass = 0; pass < 3; ++pass) {
                std::vector<char> want(og.nrhs, 0);
                bool any = false;
                int used = 0;
                for (int k = 0; k < og.nrhs; ++k) {
                    used = std::max(used, iters[k]);
                    want[k] = status[k] == LQ_OK && !(rel[k] < cp->tol);
                    any = any || want[k];
                }
                if (!any || used >= cp->maxiter) break;
                if ((rc = correction_cg(h, og, c, wp, X, B, cp->tol, 0.5, want, cp->maxiter - used, s, iters.data(),
                                        status.data())) ||
                    (rc = residual()))
                    return rc;
                for (int k = 0; k < og.nrhs; ++k) outer[k] += want[k];
            }
            for (int k = 0; k < og.nrhs; ++k)
                if (status[k] == LQ_OK && !(rel[k] < cp->tol)) status[k] = LQ_ERR_NOT_CONVERGED;
        }
    } else {
        // FP64 defect correction around a low-precision inner CG (independent
        // per right-hand side, or one block CG over all of them)
        const bool block = mode == LQ_CG_BLOCK;
        const int ip = block ? LQ_F32 : cp->inner;
        const double itol = cp->inner_tol > 0 ? cp->inner_tol : (block ? 3e-6 : default_inner_tol(ip));
        BlockCtx bctx{h, &og, nullptr, nullptr, s};
        void *bws = nullptr, *bR = nullptr, *bP = nullptr, *bQ = nullptr;
        if (block) {
            void *bt, *btmp;
            if ((rc = ensure_ws(h, WS_CG0 + 0, og.bytes(h, LQ_F32), &bR)) ||
                (rc = ensure_ws(h, WS_CG0 + 1, og.bytes(h, LQ_F32), &bP)) ||
                (rc = ensure_ws(h, WS_CG0 + 3, og.bytes(h, LQ_F32), &bQ)) ||
                (rc = ensure_ws(h, WS_CG0 + 4, og.bytes(h, LQ_F32), &bt)) ||
                (rc = ensure_ws(h, 17, block_cg_scratch_bytes(og.nrhs), &bws)) ||
                (rc = ensure_ws(h, 16, (size_t)spinor_site_bytes(LQ_F32) * h->g.Vh * og.nrhs, &btmp)))
                return rc;
            bctx.t = static_cast<char*>(bt);
            bctx.tmp = static_cast<char*>(btmp);
            const char* L;
            size_t lb;
            if ((rc = get_links(h, LQ_F32, &L, &lb, s))) return rc;
        }
        void *r64p, *ep, *rinp;
        if ((rc = ensure_ws(h, WS_CG0 + 10, og.bytes(h, LQ_F64), &r64p)) ||
            (rc = ensure_ws(h, WS_CG0 + 11, og.bytes(h, LQ_F32), &ep)) ||
            (rc = ensure_ws(h, WS_CG0 + 12, og.bytes(h, LQ_F32), &rinp)))
            return rc;
        VecRef R64 = og.ref(h, r64p, LQ_F64), E = og.ref(h, ep, LQ_F32), RIN = og.ref(h, rinp, LQ_F32);
        if (cp->x0_is_guess) {
            if (to_native(xw, x) != cudaSuccess) return LQ_ERR_CUDA;
        } else if (cudaMemsetAsync(xw, 0, og.bytes(h, LQ_F64), s) != cudaSuccess) {
            return LQ_ERR_CUDA;
        }
        std::vector<double> bb(og.nrhs), rr(og.nrhs);
        if ((rc = norms_to_host(h, og, c, B, bb.data(), s))) return rc;
        std::vector<char> conv(og.nrhs, 0), brk(og.nrhs, 0);
        std::vector<double> best(og.nrhs, 1e300);
        std::vector<int> stall(og.nrhs, 0);
        int total_inner = 0;
        bool first = !cp->x0_is_guess;
        for (int it = 0;; ++it) {
            // r = b - A x in FP64 (the first residual of a zero start is b itself)
            if (first) {
                if (launch_axpby(R64, B, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
            } else {
                CgVecs v;
                if ((rc = cg_vectors(h, og, LQ_F64, LQ_F64, WS_CG0 + 5, &v))) return rc;
                if ((rc = apply_normal(h, og, LQ_F64, v.q.ptr, X.ptr, v.t.ptr, v.tmp.ptr, s))) return rc;
                if (launch_axpby(R64, B, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess ||
                    launch_axpby(R64, v.q, -1.0, 1.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess)
                    return LQ_ERR_CUDA;
                for (int k = 0; k < og.nrhs; ++k) iters[k] += conv[k] ? 0 : 1;
            }
            first = false;
            if ((rc = norms_to_host(h, og, c, R64, rr.data(), s))) return rc;
            bool all = true;
            for (int k = 0; k < og.nrhs; ++k) {
                rel[k] = bb[k] > 0 ? std::sqrt(rr[k] / bb[k]) : std::sqrt(rr[k]);
                if (!std::isfinite(rel[k])) status[k] = LQ_ERR_NAN;
                // three restarts without progress: the inner precision cannot reach tol
                if (rel[k] < 0.5 * best[k]) {
                    best[k] = rel[k];
                    stall[k] = 0;
                } else if (++stall[k] >= 3 && !conv[k] && rel[k] >= cp->tol) {
                    status[k] = LQ_ERR_NOT_CONVERGED;
                }
                conv[k] = conv[k] || rel[k] < cp->tol || status[k] != LQ_OK;
                all = all && conv[k];
            }
            if (all) break;
            if (total_inner >= cp->maxiter) {
                for (int k = 0; k < og.nrhs; ++k)
                    if (!conv[k]) status[k] = LQ_ERR_NOT_CONVERGED;
                break;
            }
            // inner tolerance: the precision's floor itol, or less work once the outer
            // target is within reach (relative to the current residual, with margin)
            double reach = 0.5;  // the smallest reduction every unfinished right-hand side still needs
            for (int k = 0; k < og.nrhs; ++k)
                if (!conv[k] && rel[k] > 0) reach = std::min(reach, 0.5 * cp->tol / rel[k]);
            int most = 0;
            if (block) {
                // one block CG over the unfinished right-hand sides, moved to the leading
                // columns of the FP32 block (a finished or zero column would make the block
                // rank-deficient); its correction is added back column by column
                std::vector<int> cols;
                for (int k = 0; k < og.nrhs; ++k)
                    if (!conv[k]) cols.push_back(k);
                const int nb = (int)cols.size();
                auto col = [](const VecRef& v, int k) { return VecRef{v.ptr + k * v.rhs_stride, v.prec, v.rhs_stride}; };
                for (int m = 0; m < nb; ++m)
                    if (launch_axpby(col(RIN, m), col(R64, cols[m]), 1.0, 0.0, h->g.Vh, og.nblk, 1, s) != cudaSuccess)
                        return LQ_ERR_CUDA;
                if ((rc = ensure_pinned(h, sizeof(double2) * og.nrhs * og.nrhs + 64))) return rc;
                OpGeom ogb = og;
                ogb.nrhs = nb;
                bctx.og = &ogb;
                BlockCgOps ops{&bctx, block_apply, bctx.t};  // apply leaves K P in bctx.t
                int bit = 0;
                const double need = std::max(itol, reach);
                rc = block_cg(ops, E.ptr, RIN.ptr, static_cast<char*>(bR), static_cast<char*>(bP),
                              static_cast<char*>(bQ), E.rhs_stride, (long)og.nblk * h->g.Vh, nb, need,
                              cp->maxiter - total_inner, bws, static_cast<double2*>(h->pinned), s, &bit);
                if (rc) return rc;
                for (int m = 0; m < nb; ++m) {
                    if (launch_axpby(col(X, cols[m]), col(E, m), 1.0, 1.0, h->g.Vh, og.nblk, 1, s) != cudaSuccess)
                        return LQ_ERR_CUDA;
                    iters[cols[m]] += bit;
                    outer[cols[m]] += 1;
                }
                most = bit;
            } else {
                // inner solve A e = r (FP32 copy of r; finished right-hand sides get r = 0)
                if (launch_axpby(RIN, R64, 1.0, 0.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
                for (int k = 0; k < og.nrhs; ++k)
                    if (conv[k] && cudaMemsetAsync(RIN.ptr + k * RIN.rhs_stride, 0, RIN.rhs_stride, s) != cudaSuccess)
                        return LQ_ERR_CUDA;
                if (ip == LQ_F32) {
                    const double need = std::max(itol, reach);
                    if ((rc = run_cg(h, og, c, ip, E, RIN, need, cp->maxiter - total_inner, WS_CG0, s))) return rc;
                    for (int k = 0; k < og.nrhs; ++k) {
                        iters[k] += c.host[k].iter;
                        most = std::max(most, c.host[k].iter);
                        // <p, A p> not positive at the first step, with p = r != 0: A is singular on r
                        if (!conv[k] && c.host[k].status == LQ_ERR_BREAKDOWN && c.host[k].iter == 0)
                            status[k] = LQ_ERR_BREAKDOWN;
                    }
                } else {
                    // three precisions: an FP32 defect correction (cheap FP32 residuals) around
                    // the FP16/BF16 inner CG takes the correction to FP32's reach, so FP64
                    // residuals are needed only about twice per solve
                    const double need = std::max(kMiddleTol, reach);
                    if ((rc = solve_fp32_middle(h, og, c, ip, E, RIN, need, itol, cp->maxiter - total_inner, s,
                                                iters.data(), &most, brk.data())))
                        return rc;
                    for (int k = 0; k < og.nrhs; ++k)
                        if (!conv[k] && brk[k]) status[k] = LQ_ERR_BREAKDOWN;
                }
                for (int k = 0; k < og.nrhs; ++k)
                    if (!conv[k]) outer[k] += 1;
                if (launch_axpby(X, E, 1.0, 1.0, h->g.Vh, og.nblk, og.nrhs, s) != cudaSuccess) return LQ_ERR_CUDA;
            }
            total_inner += std::max(most, 1);
        }
    }
    // native working precision -> user layout
    cudaError_t e;
    if (native) e = launch_native_convert(fprec, x, wp, xw, h->g.Vh, og.nblk * og.nrhs, s);
    else e = launch_spinor_from_native(fprec, x, wp, xw, h->g, full, parity, nf, s);
    if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return LQ_ERR_CUDA;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int ret = LQ_OK;
    for (int k = 0; k < og.nrhs; ++k) {
        stats[k].iters = iters[k];
        stats[k].outer_iters = outer[k];
        stats[k].status = status[k];
        stats[k].true_rel_residual = rel[k];
        stats[k].time_ms = ms;
        if (status[k] != LQ_OK && ret == LQ_OK) ret = status[k];
    }
    return ret;
}

