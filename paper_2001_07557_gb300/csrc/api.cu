// api.cu -- the C ABI: handle life cycle, argument/layout checks, format
// conversion around the native hop kernels, and the Wilson / domain-wall apply
// calls.  Every entry point returns a status and never aborts.
#include <cstdlib>
#include <cstring>
#include <new>

#include "blas.h"
#include "handle.h"
#include "trace.h"

namespace lq {

cudaError_t launch_hop_batch(int prec, const HopArgs* args, const int* lat_off, int nlat, bool r12, bool dag, int epi,
                             int grid, cudaStream_t st, int* occ) {
    switch (prec) {
    case LQ_F32: return launch_hop_batch_f32(args, lat_off, nlat, r12, dag, epi, grid, st, occ);
    case LQ_F16: return launch_hop_batch_f16(args, lat_off, nlat, r12, dag, epi, grid, st, occ);
    case LQ_BF16: return launch_hop_batch_bf16(args, lat_off, nlat, r12, dag, epi, grid, st, occ);
    default: return cudaErrorInvalidValue;  // the FP64 hop has no batched form
    }
}

cudaError_t launch_hop(int prec, const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    switch (prec) {
    case LQ_F64: return launch_hop_f64(a, r12, dag, epi, block, st);
    case LQ_F32: return launch_hop_f32(a, r12, dag, epi, block, st);
    case LQ_F16: return launch_hop_f16(a, r12, dag, epi, block, st);
    default: return launch_hop_bf16(a, r12, dag, epi, block, st);
    }
}

int ensure_ws(lq_handle* h, int k, size_t bytes, void** out) {
    lq_handle::Buf& b = h->ws[k];
    if (b.bytes < bytes) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            b.ptr = nullptr;
            return LQ_ERR_NOMEM;
        }
        b.bytes = bytes;
    }
    *out = b.ptr;
    return LQ_OK;
}

int cached_graph_exec(lq_handle* h, const int key[4], cudaGraph_t graph, cudaGraphExec_t* exec) {
    constexpr int kSlots = (int)(sizeof(h->graphs) / sizeof(h->graphs[0]));
    lq_handle::GraphSlot* slot = nullptr;
    for (auto& g : h->graphs)
        if (g.exec && std::memcmp(g.key, key, sizeof(g.key)) == 0) slot = &g;
    if (slot) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(slot->exec, graph, &info) == cudaSuccess) {
            *exec = slot->exec;
            return LQ_OK;
        }
        cudaGetLastError();  // a different topology: instantiate anew in this slot
        cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
    } else {
        slot = &h->graphs[h->graph_next];
        h->graph_next = (h->graph_next + 1) % kSlots;
        if (slot->exec) cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
    }
    if (cudaGraphInstantiate(&slot->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        slot->exec = nullptr;
        return LQ_ERR_CUDA;
    }
    std::memcpy(slot->key, key, sizeof(slot->key));
    *exec = slot->exec;
    return LQ_OK;
}

int get_links(lq_handle* h, int prec, const char** links, size_t* link_block, cudaStream_t st) {
    const bool r12 = link_r12(h, prec);
    void*& L = h->links[prec][r12];
    const size_t lb = (size_t)link_site_bytes(prec, r12) * h->g.Vh;
    if (!L) {
        if (cudaMalloc(&L, lb * 8) != cudaSuccess) {
            cudaGetLastError();
            L = nullptr;
            return LQ_ERR_NOMEM;
        }
        cudaError_t e = launch_links_to_native(prec, r12, L, h->U_prec, h->U_sm, h->g, st);
        if (e != cudaSuccess) return LQ_ERR_CUDA;
    }
    *links = static_cast<const char*>(L);
    *link_block = lb;
    return LQ_OK;
}

// the fused output norm applies to operator outputs (diagonal / domain-wall epilogues) only
static void set_red(HopArgs& a, const lq_handle* h) {
    a.red_partial = h->red_partial;
    a.red_ticket = h->red_ticket;
    a.red_st = h->red_st;
}

static HopArgs base_args(lq_handle* h, const char* links, size_t lb) {
    HopArgs a;
    std::memset(&a, 0, sizeof(a));
    a.links = links;
    a.link_block = lb;
    a.g = h->g;
    a.skip = h->skip;
    a.skip_stride = h->skip_stride;
    a.mma = h->hop_kernel == LQ_HOP_TENSOR_CORES ? 1 : 0;
    return a;
}

int prep_wilson_full(lq_handle* h, int prec, char* out, const char* in, int nrhs, HopArgs* ap, cudaStream_t st) {
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    const size_t blk = native_block_bytes(h, prec);
    HopArgs a = base_args(h, L, lb);
    for (int p = 0; p < 2; ++p) {
        a.in[p] = in + (size_t)(1 - p) * blk;
        a.x[p] = in + (size_t)p * blk;
        a.out[p] = out + (size_t)p * blk;
    }
    a.in_rhs = a.out_rhs = a.x_rhs = 2 * blk;
    a.parity0 = 0;
    a.nparity = 2;
    a.nrhs = nrhs;
    a.c_hop = -0.5;
    a.c_diag = h->p.mass + 4.0;
    set_red(a, h);
    *ap = a;
    return LQ_OK;
}

int prep_wilson_block(lq_handle* h, int prec, char* out, const char* in, int out_parity, int nrhs, double c_hop,
                      HopArgs* ap, cudaStream_t st) {
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    const size_t blk = native_block_bytes(h, prec);
    HopArgs a = base_args(h, L, lb);
    a.in[out_parity] = in;
    a.out[out_parity] = out;
    a.in_rhs = a.out_rhs = blk;
    a.parity0 = out_parity;
    a.nparity = 1;
    a.nrhs = nrhs;
    a.c_hop = c_hop;
    *ap = a;
    return LQ_OK;
}

// second half of the Schur complement: out = a in - 1/(4a) H_eo tmp
int prep_wilson_schur2(lq_handle* h, int prec, char* out, const char* tmp, const char* in, int nrhs, HopArgs* ap,
                       cudaStream_t st) {
    const double am = h->p.mass + 4.0;
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    const size_t blk = native_block_bytes(h, prec);
    HopArgs a = base_args(h, L, lb);
    a.in[0] = tmp;
    a.out[0] = out;
    a.x[0] = in;
    a.in_rhs = a.out_rhs = a.x_rhs = blk;
    a.parity0 = 0;
    a.nparity = 1;
    a.nrhs = nrhs;
    a.c_hop = -1.0 / (4.0 * am);
    a.c_diag = am;
    set_red(a, h);
    *ap = a;
    return LQ_OK;
}

int native_wilson_full(lq_handle* h, int prec, char* out, const char* in, int nrhs, bool dag, cudaStream_t st) {
    HopArgs a;
    int rc = prep_wilson_full(h, prec, out, in, nrhs, &a, st);
    if (rc) return rc;
    return status_of(launch_hop(prec, a, link_r12(h, prec), dag, EPI_DIAG, h->hop_block[prec], st));
}

int native_wilson_block(lq_handle* h, int prec, char* out, const char* in, int out_parity, int nrhs, bool dag,
                        double c_hop, cudaStream_t st) {
    HopArgs a;
    int rc = prep_wilson_block(h, prec, out, in, out_parity, nrhs, c_hop, &a, st);
    if (rc) return rc;
    return status_of(launch_hop(prec, a, link_r12(h, prec), dag, EPI_HOP, h->hop_block[prec], st));
}

int native_wilson_schur(lq_handle* h, int prec, char* out, const char* in, char* tmp, int nrhs, bool dag,
                        cudaStream_t st) {
    // out = a in - 1/(4a) H_eo H_oe in
    int rc = native_wilson_block(h, prec, tmp, in, 1, nrhs, dag, 1.0, st);
    if (rc) return rc;
    HopArgs a;
    if ((rc = prep_wilson_schur2(h, prec, out, tmp, in, nrhs, &a, st))) return rc;
    return status_of(launch_hop(prec, a, link_r12(h, prec), dag, EPI_DIAG, h->hop_block[prec], st));
}

// Moebius domain wall, D_M = D_W(-M5) chi + psi - S psi with chi = b5 psi + c5 S psi:
//   chi = b5 psi + c5 S psi;  w = [(4-M5) b5 + 1] psi + [(4-M5) c5 - 1] S psi  (5th-dimension kernels)
//   out = -1/2 H chi + w                         (one Wilson hop launch, the Ls slices as right-hand sides)
// and D_M^dag psi = (b5 + c5 S^dag) D_W^dag psi + (1 - S^dag) psi:
//   z = (4-M5) psi - 1/2 H^dag psi;  out = b5 z + c5 S^dag z + psi - S^dag psi.
// The fused norm of the solver rides on the hop, whose per-slice partials
// fill the same slots as the Shamir operator's one group.
static int native_dwf_mobius(lq_handle* h, int prec, char* out, const char* in, bool dag, cudaStream_t st) {
    if (prec != LQ_F64 && prec != LQ_F32) return LQ_ERR_ARG;
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    const double b5 = h->p.b5, c5 = h->p.c5, d4 = 4.0 - h->p.M5, mf = h->p.mf;
    const size_t f5 = 2 * blk * (size_t)Ls;
    void *chi, *w;
    int rc;
    if ((rc = ensure_ws(h, WS_MOB, f5, &chi)) || (rc = ensure_ws(h, WS_MOB + 1, f5, &w))) return rc;
    HopArgs a;
    if (!dag) {
        if (launch_m5_lincomb(prec, chi, in, nullptr, h->g.Vh, 2, 2 * blk, Ls, b5, c5, 0, 0, mf, false, st) !=
                cudaSuccess ||
            launch_m5_lincomb(prec, w, in, nullptr, h->g.Vh, 2, 2 * blk, Ls, d4 * b5 + 1, d4 * c5 - 1, 0, 0, mf, false,
                              st) != cudaSuccess)
            return LQ_ERR_CUDA;
        if ((rc = prep_wilson_full(h, prec, out, static_cast<const char*>(chi), Ls, &a, st))) return rc;
        for (int p = 0; p < 2; ++p) {
            a.in[p] = static_cast<const char*>(chi) + (size_t)(1 - p) * blk;
            a.x[p] = static_cast<const char*>(w) + (size_t)p * blk;
            a.out[p] = out + (size_t)p * blk;
        }
        a.in_rhs = a.out_rhs = a.x_rhs = 2 * blk;
        a.c_diag = 1.0;
        a.skip_stride = 0;  // the slices of one system share the system's skip flag
        return status_of(launch_hop(prec, a, link_r12(h, prec), false, EPI_DIAG, h->hop_block[prec], st));
    }
    if ((rc = prep_wilson_full(h, prec, static_cast<char*>(chi), in, Ls, &a, st))) return rc;
    for (int p = 0; p < 2; ++p) {
        a.in[p] = in + (size_t)(1 - p) * blk;
        a.x[p] = in + (size_t)p * blk;
        a.out[p] = static_cast<char*>(chi) + (size_t)p * blk;
    }
    a.in_rhs = a.out_rhs = a.x_rhs = 2 * blk;
    a.c_diag = d4;
    a.skip_stride = 0;
    a.red_partial = nullptr;
    a.red_st = nullptr;
    if ((rc = status_of(launch_hop(prec, a, link_r12(h, prec), true, EPI_DIAG, h->hop_block[prec], st)))) return rc;
    return launch_m5_lincomb(prec, out, chi, in, h->g.Vh, 2, 2 * blk, Ls, b5, c5, 1.0, -1.0, mf, true, st) ==
                   cudaSuccess
               ? LQ_OK
               : LQ_ERR_CUDA;
}

int native_dwf(lq_handle* h, int prec, char* out, const char* in, bool dag, cudaStream_t st) {
    if (h->p.mobius) return native_dwf_mobius(h, prec, out, in, dag, st);
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    const size_t blk = native_block_bytes(h, prec);
    HopArgs a = base_args(h, L, lb);
    for (int p = 0; p < 2; ++p) {
        a.in[p] = in + (size_t)(1 - p) * blk;
        a.x[p] = in + (size_t)p * blk;
        a.out[p] = out + (size_t)p * blk;
    }
    a.in_rhs = a.out_rhs = a.x_rhs = 2 * blk;
    a.parity0 = 0;
    a.nparity = 2;
    a.nrhs = h->p.Ls;
    a.Ls = h->p.Ls;
    a.mf = h->p.mf;
    a.c_shift = -1.0;
    a.c_hop = -0.5;
    a.c_diag = 5.0 - h->p.M5;
    set_red(a, h);
    return status_of(launch_hop(prec, a, link_r12(h, prec), dag, EPI_DWF, h->hop_block[prec], st));
}

// Even-odd Moebius domain wall.  With B = b5 + c5 S the operator D_M = D_W(-M5) B + 1 - S
// splits by 4-d parity into the site-local part M5_M = alpha + beta S,
//   alpha = (4 - M5) b5 + 1,  beta = (4 - M5) c5 - 1,
// and M_eo = -1/2 H_eo B, M_oe = -1/2 H_oe B (B acts before the hop).  B and M5_M
// are polynomials in S, so they commute, and one sweep applies T = B M5_M^{-1}:
//   Mhat in_e     = M5_M in_e + 1/2 H_eo T (-1/2 H_oe B in_e)
//     chi = B in_e (5th-dimension pass);  tmp = -1/2 H_oe chi;  tmp = T tmp;
//     out = alpha in + beta S in + 1/2 H_eo tmp   (one domain-wall hop launch)
//   Mhat^dag in_e = M5_M^dag in_e + B^dag 1/2 H^dag_eo T^dag (-1/2 H^dag_oe in_e)
//     tmp = -1/2 H^dag_oe in;  tmp = T^dag tmp;  chi = 1/2 H^dag_eo tmp;
//     out = b5 chi + c5 S^dag chi + alpha in + beta S^dag in   (one 5th-dimension pass)
static bool mobius_site(const lq_handle* h, double* alpha, double* beta) {
    const double d4 = 4.0 - h->p.M5;
    *alpha = d4 * h->p.b5 + 1.0;
    *beta = d4 * h->p.c5 - 1.0;
    double p, g, c;
    return m5inv_coeffs(*alpha, *beta, h->p.mf, h->p.Ls, &p, &g, &c);
}

static int native_dwf_mobius_schur(lq_handle* h, int prec, char* out_e, const char* in_e, char* tmp, bool dag,
                                   cudaStream_t st) {
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    const double b5 = h->p.b5, c5 = h->p.c5, mf = h->p.mf;
    double alpha, beta;
    if (!mobius_site(h, &alpha, &beta)) return LQ_ERR_ARG;
    void* chi;
    int rc = ensure_ws(h, WS_MOB, blk * (size_t)Ls, &chi);
    if (rc) return rc;
    char* c = static_cast<char*>(chi);
    HopArgs a1;
    if (!dag && launch_m5_lincomb(prec, c, in_e, nullptr, h->g.Vh, 1, blk, Ls, b5, c5, 0, 0, mf, false, st) !=
                    cudaSuccess)
        return LQ_ERR_CUDA;
    if ((rc = prep_wilson_block(h, prec, tmp, dag ? in_e : c, 1, Ls, -0.5, &a1, st))) return rc;
    a1.skip_stride = 0;  // the slices of one system share the system's skip flag
    if ((rc = status_of(launch_hop(prec, a1, link_r12(h, prec), dag, EPI_HOP, h->hop_block[prec], st)))) return rc;
    if (launch_m5inv_general(prec, tmp, tmp, h->g.Vh, blk, blk, Ls, alpha, beta, mf, true, b5, c5, dag, st) !=
        cudaSuccess)
        return LQ_ERR_CUDA;
    if (dag) {
        if ((rc = prep_wilson_block(h, prec, c, tmp, 0, Ls, 0.5, &a1, st))) return rc;
        a1.skip_stride = 0;
        if ((rc = status_of(launch_hop(prec, a1, link_r12(h, prec), true, EPI_HOP, h->hop_block[prec], st))))
            return rc;
        return launch_m5_lincomb(prec, out_e, c, in_e, h->g.Vh, 1, blk, Ls, b5, c5, alpha, beta, mf, true, st) ==
                       cudaSuccess
                   ? LQ_OK
                   : LQ_ERR_CUDA;
    }
    const char* L;
    size_t lb;
    if ((rc = get_links(h, prec, &L, &lb, st))) return rc;
    HopArgs a = base_args(h, L, lb);
    a.in[0] = tmp;
    a.x[0] = in_e;
    a.out[0] = out_e;
    a.in_rhs = a.out_rhs = a.x_rhs = blk;
    a.parity0 = 0;
    a.nparity = 1;
    a.nrhs = Ls;
    a.Ls = Ls;
    a.mf = mf;
    a.c_shift = beta;
    a.c_hop = 0.5;
    a.c_diag = alpha;
    set_red(a, h);
    return status_of(launch_hop(prec, a, link_r12(h, prec), false, EPI_DWF, h->hop_block[prec], st));
}

// bhat_e = eta_e - M_eo M5_M^{-1} eta_o = eta_e + 1/2 H_eo T eta_o
static int native_dwf_mobius_prepare(lq_handle* h, int prec, char* bhat_e, const char* eta, char* tmp,
                                     cudaStream_t st) {
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    double alpha, beta;
    if (!mobius_site(h, &alpha, &beta)) return LQ_ERR_ARG;
    if (launch_m5inv_general(prec, tmp, eta + blk, h->g.Vh, blk, 2 * blk, Ls, alpha, beta, h->p.mf, true, h->p.b5,
                             h->p.c5, false, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    HopArgs a = base_args(h, L, lb);
    a.in[0] = tmp;
    a.x[0] = eta;
    a.out[0] = bhat_e;
    a.in_rhs = a.out_rhs = blk;
    a.x_rhs = 2 * blk;
    a.parity0 = 0;
    a.nparity = 1;
    a.nrhs = Ls;
    a.c_hop = 0.5;
    a.c_diag = 1.0;
    a.skip = nullptr;  // a source preparation is never skipped
    return status_of(launch_hop(prec, a, link_r12(h, prec), false, EPI_DIAG, h->hop_block[prec], st));
}

// psi_e = x_e;  psi_o = M5_M^{-1} (eta_o - M_oe x_e) = M5_M^{-1} (eta_o + 1/2 H_oe B x_e)
static int native_dwf_mobius_reconstruct(lq_handle* h, int prec, char* psi, const char* x_e, const char* eta,
                                         cudaStream_t st) {
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    double alpha, beta;
    if (!mobius_site(h, &alpha, &beta)) return LQ_ERR_ARG;
    void* chi;
    int rc = ensure_ws(h, WS_MOB, blk * (size_t)Ls, &chi);
    if (rc) return rc;
    if (launch_m5_lincomb(prec, chi, x_e, nullptr, h->g.Vh, 1, blk, Ls, h->p.b5, h->p.c5, 0, 0, h->p.mf, false, st) !=
        cudaSuccess)
        return LQ_ERR_CUDA;
    const char* L;
    size_t lb;
    if ((rc = get_links(h, prec, &L, &lb, st))) return rc;
    HopArgs a = base_args(h, L, lb);
    a.in[1] = static_cast<const char*>(chi);
    a.x[1] = eta + blk;
    a.out[1] = psi + blk;
    a.in_rhs = blk;
    a.out_rhs = a.x_rhs = 2 * blk;
    a.parity0 = 1;
    a.nparity = 1;
    a.nrhs = Ls;
    a.c_hop = 0.5;
    a.c_diag = 1.0;
    a.skip = nullptr;
    if ((rc = status_of(launch_hop(prec, a, link_r12(h, prec), false, EPI_DIAG, h->hop_block[prec], st))))
        return rc;
    if (launch_m5inv_general(prec, psi + blk, psi + blk, h->g.Vh, 2 * blk, 2 * blk, Ls, alpha, beta, h->p.mf, false,
                             1.0, 0.0, false, st) != cudaSuccess ||
        cudaMemcpy2DAsync(psi, 2 * blk, x_e, blk, blk, Ls, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    return LQ_OK;
}

// Even-odd domain wall: Mhat = M5 - M_eo M5^{-1} M_oe with M_eo = -1/2 H_eo on
// every slice (the 5th-dimension index runs as the right-hand-side index of
// the Wilson hop) and M5 the site-local part of D_dw.
//   tmp_o = -1/2 H_oe in_e;  tmp_o = M5^{-1} tmp_o;  out_e = M5 in_e + 1/2 H_eo tmp_o,
// the last as one domain-wall hop launch (its epilogue is exactly M5 in_e).
// The dagger uses the daggered hop, (M5^dag)^{-1} and M5^dag.
int native_dwf_schur(lq_handle* h, int prec, char* out_e, const char* in_e, char* tmp, bool dag, cudaStream_t st) {
    if (prec != LQ_F64 && prec != LQ_F32) return LQ_ERR_ARG;
    if (h->p.mobius) return native_dwf_mobius_schur(h, prec, out_e, in_e, tmp, dag, st);
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    HopArgs a1;
    int rc = prep_wilson_block(h, prec, tmp, in_e, 1, Ls, -0.5, &a1, st);
    if (rc) return rc;
    a1.skip_stride = 0;  // the slices of one system share the system's skip flag
    if ((rc = status_of(launch_hop(prec, a1, link_r12(h, prec), dag, EPI_HOP, h->hop_block[prec], st)))) return rc;
    if (launch_m5inv(prec, tmp, tmp, h->g.Vh, blk, blk, Ls, h->p.M5, h->p.mf, dag, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    const char* L;
    size_t lb;
    if ((rc = get_links(h, prec, &L, &lb, st))) return rc;
    HopArgs a = base_args(h, L, lb);
    a.in[0] = tmp;
    a.x[0] = in_e;
    a.out[0] = out_e;
    a.in_rhs = a.out_rhs = a.x_rhs = blk;
    a.parity0 = 0;
    a.nparity = 1;
    a.nrhs = Ls;
    a.Ls = Ls;
    a.mf = h->p.mf;
    a.c_shift = -1.0;
    a.c_hop = 0.5;
    a.c_diag = 5.0 - h->p.M5;
    set_red(a, h);
    return status_of(launch_hop(prec, a, link_r12(h, prec), dag, EPI_DWF, h->hop_block[prec], st));
}

// bhat_e = eta_e - M_eo M5^{-1} eta_o = eta_e + 1/2 H_eo M5^{-1} eta_o  (eta a full 5-d field)
int native_dwf_prepare(lq_handle* h, int prec, char* bhat_e, const char* eta, char* tmp, cudaStream_t st) {
    if (prec != LQ_F64 && prec != LQ_F32) return LQ_ERR_ARG;
    if (h->p.mobius) return native_dwf_mobius_prepare(h, prec, bhat_e, eta, tmp, st);
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    if (launch_m5inv(prec, tmp, eta + blk, h->g.Vh, blk, 2 * blk, Ls, h->p.M5, h->p.mf, false, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    HopArgs a = base_args(h, L, lb);
    a.in[0] = tmp;
    a.x[0] = eta;
    a.out[0] = bhat_e;
    a.in_rhs = a.out_rhs = blk;
    a.x_rhs = 2 * blk;
    a.parity0 = 0;
    a.nparity = 1;
    a.nrhs = Ls;
    a.c_hop = 0.5;
    a.c_diag = 1.0;
    a.skip = nullptr;  // a source preparation is never skipped
    return status_of(launch_hop(prec, a, link_r12(h, prec), false, EPI_DIAG, h->hop_block[prec], st));
}

// psi_e = x_e;  psi_o = M5^{-1} (eta_o - M_oe x_e) = M5^{-1} (eta_o + 1/2 H_oe x_e)
int native_dwf_reconstruct(lq_handle* h, int prec, char* psi, const char* x_e, const char* eta, cudaStream_t st) {
    if (prec != LQ_F64 && prec != LQ_F32) return LQ_ERR_ARG;
    if (h->p.mobius) return native_dwf_mobius_reconstruct(h, prec, psi, x_e, eta, st);
    const int Ls = h->p.Ls;
    const size_t blk = native_block_bytes(h, prec);
    const char* L;
    size_t lb;
    int rc = get_links(h, prec, &L, &lb, st);
    if (rc) return rc;
    HopArgs a = base_args(h, L, lb);
    a.in[1] = x_e;
    a.x[1] = eta + blk;
    a.out[1] = psi + blk;
    a.in_rhs = blk;
    a.out_rhs = a.x_rhs = 2 * blk;
    a.parity0 = 1;
    a.nparity = 1;
    a.nrhs = Ls;
    a.c_hop = 0.5;
    a.c_diag = 1.0;
    a.skip = nullptr;
    if ((rc = status_of(launch_hop(prec, a, link_r12(h, prec), false, EPI_DIAG, h->hop_block[prec], st))))
        return rc;
    if (launch_m5inv(prec, psi + blk, psi + blk, h->g.Vh, 2 * blk, 2 * blk, Ls, h->p.M5, h->p.mf, false, st) !=
            cudaSuccess ||
        cudaMemcpy2DAsync(psi, 2 * blk, x_e, blk, blk, Ls, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    return LQ_OK;
}

}  // namespace lq

using namespace lq;

namespace {

int wilson_apply(lq_handle* h, void* out, const void* in, int fmt, int parity, int nrhs, cudaStream_t st,
                 bool dag) {
    if (!h || !out || !in) return LQ_ERR_ARG;
    if (!valid_fmt(fmt) || nrhs < 1) return LQ_ERR_ARG;
    if (parity < LQ_FULL || parity > LQ_SCHUR_EVEN) return LQ_ERR_ARG;
    if (!aligned16(out) || !aligned16(in)) return LQ_ERR_LAYOUT;
    const int subset = parity == LQ_FULL ? LQ_FULL : LQ_EVEN;
    const size_t nb = field_bytes(h, fmt, subset, nrhs);
    if (overlap(out, nb, in, nb)) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    const int prec = fmt & 0xF;
    const bool native = (fmt & LQ_NATIVE) != 0;
    const bool full = parity == LQ_FULL;
    const int in_par = parity == LQ_FULL ? 0 : parity == LQ_SCHUR_EVEN ? 0 : 1 - parity;
    const int out_par = parity == LQ_FULL ? 0 : parity == LQ_SCHUR_EVEN ? 0 : parity;
    const size_t nat = field_bytes(h, prec | LQ_NATIVE, subset, nrhs);
    const char* nin = static_cast<const char*>(in);
    char* nout = static_cast<char*>(out);
    int rc;
    if (!native) {
        void *a, *b;
        if ((rc = ensure_ws(h, WS_IN, nat, &a)) || (rc = ensure_ws(h, WS_OUT, nat, &b))) return rc;
        if (launch_spinor_to_native(prec, a, prec, in, h->g, full, in_par, nrhs, st) != cudaSuccess)
            return LQ_ERR_CUDA;
        nin = static_cast<const char*>(a);
        nout = static_cast<char*>(b);
    }
    if (parity == LQ_FULL) {
        rc = native_wilson_full(h, prec, nout, nin, nrhs, dag, st);
    } else if (parity == LQ_SCHUR_EVEN) {
        void* t;
        if ((rc = ensure_ws(h, WS_TMP, nat, &t))) return rc;
        rc = native_wilson_schur(h, prec, nout, nin, static_cast<char*>(t), nrhs, dag, st);
    } else {
        rc = native_wilson_block(h, prec, nout, nin, parity, nrhs, dag, -0.5, st);
    }
    if (rc) return rc;
    if (!native) {
        if (launch_spinor_from_native(prec, out, prec, nout, h->g, full, out_par, nrhs, st) != cudaSuccess)
            return LQ_ERR_CUDA;
    }
    return LQ_OK;
}

}  // namespace

extern "C" {

// Largest deviation from SU(3) (|U^dag U - 1| entry, |det U - 1|) accepted for
// two-row link storage: FP64 links are unitary to ~1e-15, FP32 ones to ~1e-7.
constexpr double kSu3TolF64 = 1e-6, kSu3TolF32 = 1e-5;

int lq_create(lq_handle** hp, const lq_params* p, const void* U, int U_prec, void* stream) {
    lq::TraceRange trace_("lqcd/create");
    if (!hp || !p || !U) return LQ_ERR_ARG;
    *hp = nullptr;
    if (U_prec != LQ_F64 && U_prec != LQ_F32) return LQ_ERR_ARG;
    if (!aligned16(U)) return LQ_ERR_LAYOUT;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (p->dims[mu] < 2 || (p->dims[mu] & 1) || p->dims[mu] > 8192) return LQ_ERR_LAYOUT;
        if (p->bc[mu] != 1 && p->bc[mu] != -1) return LQ_ERR_ARG;
        V *= p->dims[mu];
    }
    if (V / 2 >= (1LL << 27)) return LQ_ERR_LAYOUT;  // cb indices < 2^27: exact fast division
    if (p->r != 1.0) return LQ_ERR_ARG;
    if (p->Ls < 0 || p->Ls > 4096) return LQ_ERR_ARG;
    if (p->mobius && (p->mobius != 1 || p->Ls < 1)) return LQ_ERR_ARG;
    lq_handle* h = new (std::nothrow) lq_handle;
    if (!h) return LQ_ERR_NOMEM;
    std::memset(h, 0, sizeof(*h));
    h->p = *p;
    for (int mu = 0; mu < 4; ++mu) {
        h->g.L[mu] = p->dims[mu];
        h->g.bc[mu] = p->bc[mu];
    }
    h->g.Lh0 = p->dims[0] / 2;
    h->g.Vh = (int)(V / 2);
    h->g.mLh0 = div_magic(h->g.Lh0);
    h->g.mL1 = div_magic(p->dims[1]);
    h->g.mL2 = div_magic(p->dims[2]);
    for (int k = 0; k < 4; ++k) h->hop_block[k] = kHopThreads;
    h->hop_kernel = LQ_HOP_CUDA_CORES;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return LQ_ERR_CUDA;
    }
    h->U_prec = U_prec;
    const size_t ub = (size_t)V * 72 * (U_prec == LQ_F64 ? 8 : 4);
    if (cudaMalloc(&h->U_sm, ub) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LQ_ERR_NOMEM;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h->U_sm, U, ub, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        lq_destroy(h);
        return LQ_ERR_CUDA;
    }
    if (p->compress12) {
        // two-row storage rebuilds row 3 from rows 1 and 2, exact only for SU(3) links:
        // a link further from SU(3) than the input precision's rounding allows is refused
        double dev = 0.0;
        if (link_su3_deviation(U_prec, h->U_sm, V * 4, &dev, st) != cudaSuccess) {
            lq_destroy(h);
            return LQ_ERR_CUDA;
        }
        if (!(dev <= (U_prec == LQ_F64 ? kSu3TolF64 : kSu3TolF32))) {
            lq_destroy(h);
            return LQ_ERR_ARG;
        }
    }
    *hp = h;
    return LQ_OK;
}

int lq_destroy(lq_handle* h) {
    if (!h) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    if (h->U_sm) cudaFree(h->U_sm);
    for (auto& l : h->links)
        for (void* q : l)
            if (q) cudaFree(q);
    for (auto& b : h->ws)
        if (b.ptr) cudaFree(b.ptr);
    for (auto& g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->solver_stream) cudaStreamDestroy(h->solver_stream);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
    return LQ_OK;
}

int lq_field_bytes(const lq_handle* h, int fmt, int subset, int nrhs, int five_d, size_t* bytes) {
    if (!h || !bytes || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (subset < LQ_FULL || subset > LQ_ODD) return LQ_ERR_ARG;
    if (five_d) {
        if (h->p.Ls < 1) return LQ_ERR_ARG;
        *bytes = field_bytes(h, fmt, LQ_FULL, h->p.Ls);
        return LQ_OK;
    }
    if (nrhs < 1) return LQ_ERR_ARG;
    *bytes = field_bytes(h, fmt, subset, nrhs);
    return LQ_OK;
}

int lq_convert(lq_handle* h, void* dst, int dst_fmt, const void* src, int src_fmt, int subset, int nrhs, int five_d,
               void* stream) {
    lq::TraceRange trace_("lqcd/convert");
    if (!h || !dst || !src || !valid_fmt(dst_fmt) || !valid_fmt(src_fmt)) return LQ_ERR_ARG;
    if (subset < LQ_FULL || subset > LQ_ODD) return LQ_ERR_ARG;
    if (!aligned16(dst) || !aligned16(src)) return LQ_ERR_LAYOUT;
    {
        DeviceGuard dg(h->device);
        if (!device_accessible(dst) || !device_accessible(src)) return LQ_ERR_LAYOUT;
    }
    if (five_d) {
        if (h->p.Ls < 1) return LQ_ERR_ARG;
        subset = LQ_FULL;
        nrhs = h->p.Ls;
    }
    if (nrhs < 1) return LQ_ERR_ARG;
    if (overlap(dst, field_bytes(h, dst_fmt, subset, nrhs), src, field_bytes(h, src_fmt, subset, nrhs)))
        return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool full = subset == LQ_FULL;
    const int parity = full ? 0 : subset;
    const int dp = dst_fmt & 0xF, sp = src_fmt & 0xF;
    const bool dn = (dst_fmt & LQ_NATIVE) != 0, sn = (src_fmt & LQ_NATIVE) != 0;
    cudaError_t e;
    if (dn && sn) {
        e = launch_native_convert(dp, dst, sp, src, h->g.Vh, nrhs * (full ? 2 : 1), st);
    } else if (dn && !sn) {
        e = launch_spinor_to_native(dp, dst, sp, src, h->g, full, parity, nrhs, st);
    } else if (!dn && sn) {
        e = launch_spinor_from_native(dp, dst, sp, src, h->g, full, parity, nrhs, st);
    } else {
        // site-major -> site-major precision change goes through a native FP64 copy
        void* t;
        int rc = ensure_ws(h, WS_IN, field_bytes(h, LQ_F64 | LQ_NATIVE, subset, nrhs), &t);
        if (rc) return rc;
        e = launch_spinor_to_native(LQ_F64, t, sp, src, h->g, full, parity, nrhs, st);
        if (e == cudaSuccess) e = launch_spinor_from_native(dp, dst, LQ_F64, t, h->g, full, parity, nrhs, st);
    }
    return status_of(e);
}

int dslash_apply(lq_handle* h, void* out, const void* in, int fmt, int parity, int nrhs, void* stream) {
    lq::TraceRange trace_("lqcd/dslash");
    return wilson_apply(h, out, in, fmt, parity, nrhs, static_cast<cudaStream_t>(stream), false);
}

int dslash_dag_apply(lq_handle* h, void* out, const void* in, int fmt, int parity, int nrhs, void* stream) {
    lq::TraceRange trace_("lqcd/dslash_dag");
    return wilson_apply(h, out, in, fmt, parity, nrhs, static_cast<cudaStream_t>(stream), true);
}

int dwf_dslash_apply(lq_handle* h, void* out, const void* in, int fmt, int dagger, void* stream) {
    lq::TraceRange trace_("lqcd/dwf_dslash");
    if (!h || !out || !in || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (h->p.Ls < 1) return LQ_ERR_ARG;
    if (!aligned16(out) || !aligned16(in)) return LQ_ERR_LAYOUT;
    const size_t nb = field_bytes(h, fmt, LQ_FULL, h->p.Ls);
    if (overlap(out, nb, in, nb)) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int prec = fmt & 0xF;
    const bool native = (fmt & LQ_NATIVE) != 0;
    const int Ls = h->p.Ls;
    const char* nin = static_cast<const char*>(in);
    char* nout = static_cast<char*>(out);
    int rc;
    if (!native) {
        const size_t nat = field_bytes(h, prec | LQ_NATIVE, LQ_FULL, Ls);
        void *a, *b;
        if ((rc = ensure_ws(h, WS_IN, nat, &a)) || (rc = ensure_ws(h, WS_OUT, nat, &b))) return rc;
        if (launch_spinor_to_native(prec, a, prec, in, h->g, true, 0, Ls, st) != cudaSuccess) return LQ_ERR_CUDA;
        nin = static_cast<const char*>(a);
        nout = static_cast<char*>(b);
    }
    rc = native_dwf(h, prec, nout, nin, dagger != 0, st);
    if (rc) return rc;
    if (!native) {
        if (launch_spinor_from_native(prec, out, prec, nout, h->g, true, 0, Ls, st) != cudaSuccess)
            return LQ_ERR_CUDA;
    }
    return LQ_OK;
}

// Even-odd domain wall (Shamir or Moebius): argument checks shared by the three calls (FP64/FP32 only).
static int dwf_eo_args(lq_handle* h, int fmt) {
    if (!h || !valid_fmt(fmt)) return LQ_ERR_ARG;
    const int prec = fmt & 0xF;
    if (h->p.Ls < 1 || (prec != LQ_F64 && prec != LQ_F32)) return LQ_ERR_ARG;
    return LQ_OK;
}

int dwf_schur_apply(lq_handle* h, void* out, const void* in, int fmt, int dagger, void* stream) {
    lq::TraceRange trace_("lqcd/dwf_schur");
    int rc = dwf_eo_args(h, fmt);
    if (rc) return rc;
    if (!out || !in) return LQ_ERR_ARG;
    if (!aligned16(out) || !aligned16(in)) return LQ_ERR_LAYOUT;
    const int Ls = h->p.Ls, prec = fmt & 0xF;
    const size_t nb = field_bytes(h, fmt, LQ_EVEN, Ls);
    if (overlap(out, nb, in, nb)) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool native = (fmt & LQ_NATIVE) != 0;
    const size_t nat = field_bytes(h, prec | LQ_NATIVE, LQ_EVEN, Ls);
    void* tmp;
    if ((rc = ensure_ws(h, WS_TMP, nat, &tmp))) return rc;
    const char* nin = static_cast<const char*>(in);
    char* nout = static_cast<char*>(out);
    if (!native) {
        void *a, *b;
        if ((rc = ensure_ws(h, WS_IN, nat, &a)) || (rc = ensure_ws(h, WS_OUT, nat, &b))) return rc;
        if (launch_spinor_to_native(prec, a, prec, in, h->g, false, LQ_EVEN, Ls, st) != cudaSuccess)
            return LQ_ERR_CUDA;
        nin = static_cast<const char*>(a);
        nout = static_cast<char*>(b);
    }
    if ((rc = native_dwf_schur(h, prec, nout, nin, static_cast<char*>(tmp), dagger != 0, st))) return rc;
    if (!native && launch_spinor_from_native(prec, out, prec, nout, h->g, false, LQ_EVEN, Ls, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    return LQ_OK;
}

int dwf_eo_prepare(lq_handle* h, void* bhat_e, const void* eta, int fmt, void* stream) {
    lq::TraceRange trace_("lqcd/dwf_eo_prepare");
    int rc = dwf_eo_args(h, fmt);
    if (rc) return rc;
    if (!bhat_e || !eta) return LQ_ERR_ARG;
    if (!aligned16(bhat_e) || !aligned16(eta)) return LQ_ERR_LAYOUT;
    const int Ls = h->p.Ls, prec = fmt & 0xF;
    if (overlap(bhat_e, field_bytes(h, fmt, LQ_EVEN, Ls), eta, field_bytes(h, fmt, LQ_FULL, Ls))) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool native = (fmt & LQ_NATIVE) != 0;
    void* tmp;
    if ((rc = ensure_ws(h, WS_TMP, field_bytes(h, prec | LQ_NATIVE, LQ_EVEN, Ls), &tmp))) return rc;
    const char* neta = static_cast<const char*>(eta);
    char* nb = static_cast<char*>(bhat_e);
    if (!native) {
        void *a, *b;
        if ((rc = ensure_ws(h, WS_IN, field_bytes(h, prec | LQ_NATIVE, LQ_FULL, Ls), &a)) ||
            (rc = ensure_ws(h, WS_OUT, field_bytes(h, prec | LQ_NATIVE, LQ_EVEN, Ls), &b)))
            return rc;
        if (launch_spinor_to_native(prec, a, prec, eta, h->g, true, 0, Ls, st) != cudaSuccess) return LQ_ERR_CUDA;
        neta = static_cast<const char*>(a);
        nb = static_cast<char*>(b);
    }
    if ((rc = native_dwf_prepare(h, prec, nb, neta, static_cast<char*>(tmp), st))) return rc;
    if (!native && launch_spinor_from_native(prec, bhat_e, prec, nb, h->g, false, LQ_EVEN, Ls, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    return LQ_OK;
}

int dwf_eo_reconstruct(lq_handle* h, void* psi, const void* x_e, const void* eta, int fmt, void* stream) {
    lq::TraceRange trace_("lqcd/dwf_eo_reconstruct");
    int rc = dwf_eo_args(h, fmt);
    if (rc) return rc;
    if (!psi || !x_e || !eta) return LQ_ERR_ARG;
    if (!aligned16(psi) || !aligned16(x_e) || !aligned16(eta)) return LQ_ERR_LAYOUT;
    const int Ls = h->p.Ls, prec = fmt & 0xF;
    const size_t full = field_bytes(h, fmt, LQ_FULL, Ls), half = field_bytes(h, fmt, LQ_EVEN, Ls);
    if (overlap(psi, full, x_e, half) || overlap(psi, full, eta, full)) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool native = (fmt & LQ_NATIVE) != 0;
    const char* nx = static_cast<const char*>(x_e);
    const char* neta = static_cast<const char*>(eta);
    char* npsi = static_cast<char*>(psi);
    if (!native) {
        void *a, *b, *c;
        if ((rc = ensure_ws(h, WS_IN, field_bytes(h, prec | LQ_NATIVE, LQ_EVEN, Ls), &a)) ||
            (rc = ensure_ws(h, WS_TMP, field_bytes(h, prec | LQ_NATIVE, LQ_FULL, Ls), &b)) ||
            (rc = ensure_ws(h, WS_OUT, field_bytes(h, prec | LQ_NATIVE, LQ_FULL, Ls), &c)))
            return rc;
        if (launch_spinor_to_native(prec, a, prec, x_e, h->g, false, LQ_EVEN, Ls, st) != cudaSuccess ||
            launch_spinor_to_native(prec, b, prec, eta, h->g, true, 0, Ls, st) != cudaSuccess)
            return LQ_ERR_CUDA;
        nx = static_cast<const char*>(a);
        neta = static_cast<const char*>(b);
        npsi = static_cast<char*>(c);
    }
    if ((rc = native_dwf_reconstruct(h, prec, npsi, nx, neta, st))) return rc;
    if (!native && launch_spinor_from_native(prec, psi, prec, npsi, h->g, true, 0, Ls, st) != cudaSuccess)
        return LQ_ERR_CUDA;
    return LQ_OK;
}

int lq_dot(lq_handle* h, double* result, const void* a, const void* b, int fmt, int subset, int nrhs, int five_d,
           void* stream) {
    lq::TraceRange trace_("lqcd/dot");
    if (!h || !result || !a || !b || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (subset < LQ_FULL || subset > LQ_ODD) return LQ_ERR_ARG;
    if (!aligned16(a) || !aligned16(b) || (reinterpret_cast<uintptr_t>(result) & 7u)) return LQ_ERR_LAYOUT;
    long nsites;
    if (five_d) {
        if (h->p.Ls < 1) return LQ_ERR_ARG;
        nrhs = 1;
        nsites = 2L * h->g.Vh * h->p.Ls;
    } else {
        if (nrhs < 1) return LQ_ERR_ARG;
        nsites = (subset == LQ_FULL ? 2L : 1L) * h->g.Vh;
    }
    if (nrhs > 65535) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    if (!device_accessible(result) || !device_accessible(a) || !device_accessible(b)) return LQ_ERR_LAYOUT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool native = (fmt & LQ_NATIVE) != 0;
    const int prec = fmt & 0xF;
    const size_t site_bytes = native ? (size_t)spinor_site_bytes(prec) : (size_t)24 * (prec == LQ_F64 ? 8 : 4);
    void* ws;
    const size_t nb = sizeof(double) * 2 * kMaxGrid * (size_t)nrhs + sizeof(unsigned) * nrhs;
    int rc = ensure_ws(h, WS_DOT, nb, &ws);
    if (rc) return rc;
    double* partial = static_cast<double*>(ws);
    unsigned* tickets = reinterpret_cast<unsigned*>(partial + 2 * kMaxGrid * (size_t)nrhs);
    if (cudaMemsetAsync(tickets, 0, sizeof(unsigned) * nrhs, st) != cudaSuccess) return LQ_ERR_CUDA;
    return status_of(launch_cdot(fmt, a, b, site_bytes * nsites, nsites, h->g.Vh, nrhs, partial, tickets, result, st));
}

int lq_index_faults(unsigned long long* count, long long* first, int* checked) {
    if (!count) return LQ_ERR_ARG;
#ifdef LQ_INDEX_CHECK
    const int on = 1;
#else
    const int on = 0;
#endif
    if (checked) *checked = on;
    if (first) *first = -1;
    unsigned long long total = 0;
    for (auto rd : {index_faults_f64, index_faults_f32, index_faults_f16, index_faults_bf16}) {
        long long f = -1;
        const unsigned long long c = rd(&f);
        if (c == ~0ull) return LQ_ERR_CUDA;
        if (c && first && *first < 0) *first = f;
        total += c;
    }
    *count = total;
    return LQ_OK;
}

int lq_set_hop_kernel(lq_handle* h, int kind) {
    if (!h || (kind != LQ_HOP_CUDA_CORES && kind != LQ_HOP_TENSOR_CORES)) return LQ_ERR_ARG;
    h->hop_kernel = kind;
    return LQ_OK;
}

const char* lq_status_string(int status) {
    switch (status) {
    case LQ_OK: return "ok";
    case LQ_ERR_ARG: return "invalid argument";
    case LQ_ERR_LAYOUT: return "unsupported layout or misaligned pointer";
    case LQ_ERR_CUDA: return "CUDA error";
    case LQ_ERR_NOMEM: return "out of device memory";
    case LQ_ERR_NOT_CONVERGED: return "solver did not converge";
    case LQ_ERR_BREAKDOWN: return "solver breakdown";
    case LQ_ERR_TIMEOUT: return "device-side wait timed out";
    case LQ_ERR_NAN: return "NaN or Inf encountered";
    default: return "unknown status";
    }
}

}  // extern "C"
