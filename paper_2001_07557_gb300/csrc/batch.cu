// batch.cu -- lq_batch_cg_solve: CG on several independent lattices of
// different sizes at once (each with nrhs right-hand sides).
//
// Every operator application of the iteration is ONE persistent launch that
// walks the work items of all lattices (wilson_hop_batch_kernel), and every
// vector step is one launch over a table of (lattice, right-hand side)
// segments; the whole iteration is captured once into a CUDA graph and
// replayed.  The persistent launch's shape -- sites per work item (a multiple
// of the 128-thread tile) and the number of resident blocks -- comes from the
// library's autotuner, which times the candidates on the actual batch once and
// remembers the winner per batch shape (in memory, and in the file named by
// LQCD_TUNE_CACHE when that is set).
//
// The solve is the FP64 defect correction of cg.cu (FP64 solution and true
// residuals per lattice; inner CG with p, A p in the inner storage precision
// and the iterate and residual in FP32), with an FP32 middle level between
// the two for FP16/BF16 inner precisions, or a plain FP32 CG.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "blas.h"
#include "handle.h"
#include "trace.h"

namespace lq {

namespace {

constexpr int kIters = 8;  // iterations per graph replay
constexpr double kMiddleTolBatch = 1e-5;  // the FP32 middle level's target, as in cg.cu

// A launch shape of the persistent hop: 128-site tiles per work item of each
// lattice, and resident blocks.
struct Tune {
    std::vector<int> mult;
    int grid;
};

std::mutex g_tune_mutex;
std::map<std::string, Tune> g_tune;
bool g_tune_file_loaded = false;

// Cache file (LQCD_TUNE_CACHE): one line per batch shape,
//   <key> <grid> <nlat> <mult of lattice 0> ... <mult of lattice nlat-1>
void tune_file_load() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char* path = getenv("LQCD_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[512];
    int gr, n;
    while (fscanf(f, "%511s %d %d", key, &gr, &n) == 3 && n >= 1 && n <= 64) {
        Tune tu{std::vector<int>(n), gr};
        bool ok = true;
        for (int l = 0; l < n && ok; ++l) ok = fscanf(f, "%d", &tu.mult[l]) == 1 && tu.mult[l] >= 1;
        if (!ok) break;
        g_tune[key] = tu;
    }
    fclose(f);
}

void tune_file_save() {
    const char* path = getenv("LQCD_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_tune) {
        fprintf(f, "%s %d %d", kv.first.c_str(), kv.second.grid, (int)kv.second.mult.size());
        for (int m : kv.second.mult) fprintf(f, " %d", m);
        fprintf(f, "\n");
    }
    fclose(f);
}

struct Lat {
    lq_handle* h;
    int nblk;      // parity blocks per right-hand side
    int subset;    // LQ_FULL / LQ_EVEN
    size_t b64, b32, bp;  // bytes of one nrhs field in FP64, FP32, inner precision
    char *X64, *B64, *R64, *E, *RIN, *r, *p, *q, *t, *tmp, *tmp2;  // native fields
    char *q64, *t64, *tmp64;
    char *RIN0, *EM, *q32, *t32, *tmp32;  // FP32 middle level (16-bit inner precisions)
};

int alloc_lat(Lat& L, int op, int nr, int ip) {
    lq_handle* h = L.h;
    L.nblk = op == LQ_OP_WILSON_NORMAL ? 2 : 1;
    L.subset = op == LQ_OP_WILSON_NORMAL ? LQ_FULL : LQ_EVEN;
    const size_t Vh = h->g.Vh;
    L.b64 = (size_t)L.nblk * spinor_site_bytes(LQ_F64) * Vh * nr;
    L.b32 = (size_t)L.nblk * spinor_site_bytes(LQ_F32) * Vh * nr;
    L.bp = (size_t)L.nblk * spinor_site_bytes(ip) * Vh * nr;
    const size_t half_p = (size_t)spinor_site_bytes(ip) * Vh * nr, half64 = (size_t)spinor_site_bytes(LQ_F64) * Vh * nr;
    struct {
        char** ptr;
        size_t n;
    } want[] = {{&L.B64, L.b64},  {&L.X64, L.b64}, {&L.R64, L.b64},  {&L.E, L.b32},   {&L.RIN, L.b32},
                {&L.r, L.b32},    {&L.p, L.bp},    {&L.q, L.bp},     {&L.t, L.bp},    {&L.tmp, half_p},
                {&L.tmp2, half_p}, {&L.q64, L.b64}, {&L.t64, L.b64}, {&L.tmp64, half64}};
    int slot = 0;
    for (auto& w : want) {
        void* p;
        int rc = ensure_ws(h, slot++, w.n, &p);
        if (rc) return rc;
        *w.ptr = static_cast<char*>(p);
    }
    L.RIN0 = L.EM = L.q32 = L.t32 = L.tmp32 = nullptr;
    if (ip == LQ_F16 || ip == LQ_BF16) {
        const size_t half32 = (size_t)spinor_site_bytes(LQ_F32) * Vh * nr;
        struct {
            char** ptr;
            size_t n;
            int slot;
        } mid[] = {{&L.RIN0, L.b32, 14}, {&L.EM, L.b32, 15}, {&L.q32, L.b32, 16}, {&L.t32, L.b32, 17},
                   {&L.tmp32, half32, 20}};
        for (auto& w : mid) {
            void* p;
            int rc = ensure_ws(h, w.slot, w.n, &p);
            if (rc) return rc;
            *w.ptr = static_cast<char*>(p);
        }
    }
    return LQ_OK;
}

// out = K^dag K in for one lattice (used for the FP64 residuals)
int apply_normal_one(Lat& L, int op, int prec, char* out, const char* in, char* t, char* tmp, int nr, cudaStream_t s) {
    int rc;
    if (op == LQ_OP_WILSON_NORMAL) {
        if ((rc = native_wilson_full(L.h, prec, t, in, nr, false, s))) return rc;
        return native_wilson_full(L.h, prec, out, t, nr, true, s);
    }
    if ((rc = native_wilson_schur(L.h, prec, t, in, tmp, nr, false, s))) return rc;
    return native_wilson_schur(L.h, prec, out, t, tmp, nr, true, s);
}

}  // namespace

}  // namespace lq

using namespace lq;

extern "C" int lq_batch_cg_solve(lq_handle** hs, int nlat, void** xs, const void** bs, const lq_cg_params* cp,
                                 lq_cg_stats* stats, void* stream) {
    lq::TraceRange trace_("lqcd/batch_cg_solve");
    if (!hs || !xs || !bs || !cp || !stats || nlat < 1 || nlat > 64) return LQ_ERR_ARG;
    if (cp->op != LQ_OP_WILSON_NORMAL && cp->op != LQ_OP_WILSON_EO_NORMAL) return LQ_ERR_ARG;
    if (cp->nrhs < 1 || cp->nrhs > 64 || cp->maxiter < 1 || !(cp->tol > 0) || !valid_fmt(cp->fmt)) return LQ_ERR_ARG;
    const int mode = cp->mode == LQ_CG_BATCHED ? LQ_CG_MIXED : cp->mode;
    const int fprec = cp->fmt & 0xF;
    const bool native = (cp->fmt & LQ_NATIVE) != 0;
    if (fprec > LQ_F32) return LQ_ERR_ARG;
    int ip;  // precision of p and A p
    if (mode == LQ_CG_MIXED) {
        if (cp->inner < LQ_F32 || cp->inner > LQ_BF16) return LQ_ERR_ARG;
        ip = cp->inner;
    } else if (mode == LQ_CG_PLAIN && fprec == LQ_F32) {
        ip = LQ_F32;
    } else {
        return LQ_ERR_ARG;  // the batched operator runs in FP32 / FP16 / BF16 storage
    }
    const int nr = cp->nrhs;
    for (int l = 0; l < nlat; ++l) {
        if (!hs[l] || !xs[l] || !bs[l]) return LQ_ERR_ARG;
        if (!aligned16(xs[l]) || !aligned16(bs[l])) return LQ_ERR_LAYOUT;
        if (hs[l]->device != hs[0]->device || hs[l]->p.compress12 != hs[0]->p.compress12) return LQ_ERR_ARG;
        for (int m = 0; m < l; ++m)
            if (hs[m] == hs[l]) return LQ_ERR_ARG;  // one handle per lattice (workspaces are per handle)
    }
    DeviceGuard dg(hs[0]->device);
    const auto t0 = std::chrono::steady_clock::now();
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return LQ_ERR_CUDA;
    lq_handle* h0 = hs[0];
    if (!h0->solver_stream && cudaStreamCreateWithFlags(&h0->solver_stream, cudaStreamNonBlocking) != cudaSuccess)
        return LQ_ERR_CUDA;
    cudaStream_t s = h0->solver_stream;
    const bool r12 = h0->p.compress12 != 0;
    const int op = cp->op;
    const bool mixed = mode == LQ_CG_MIXED;
    const int wp = mixed ? LQ_F64 : LQ_F32;  // precision of x and b inside the solver

    std::vector<Lat> lat(nlat);
    int rc;
    for (int l = 0; l < nlat; ++l) {
        lat[l].h = hs[l];
        if ((rc = alloc_lat(lat[l], op, nr, ip))) return rc;
        const char* L;
        size_t lb;
        if ((rc = get_links(hs[l], ip, &L, &lb, s)) || (mixed && (rc = get_links(hs[l], LQ_F64, &L, &lb, s))) ||
            (mixed && ip != LQ_F32 && (rc = get_links(hs[l], LQ_F32, &L, &lb, s))))
            return rc;
    }
    // solver state of all (lattice, rhs) segments: scalars, tables, partials (first handle's workspace)
    const int nseg = nlat * nr;
    long maxsites = 0;
    for (auto& L : lat) maxsites = std::max(maxsites, (long)L.nblk * L.h->g.Vh);
    const int gx = (int)std::max(1L, std::min((maxsites + 255) / 256, (long)std::max(1, 1216 / nseg)));
    const int nhopk = op == LQ_OP_WILSON_NORMAL ? 2 : 4;  // hop launches per operator application
    size_t npart = (size_t)gx * nseg;  // batched reductions, and the per-lattice norms
    for (auto& L : lat) npart = std::max(npart, reduce_scratch_doubles(L.h->g.Vh, L.nblk, nr));
    const size_t need = sizeof(CgScalars) * nseg + sizeof(BSeg) * nseg + sizeof(HopArgs) * nhopk * nlat +
                        sizeof(int) * 2 * (nlat + 1) + sizeof(double) * (npart + 2 * nseg) +
                        sizeof(unsigned) * nseg + 8 * 256;
    void* wsp;
    if ((rc = ensure_ws(h0, WS_CTL, need, &wsp))) return rc;
    char* q = static_cast<char*>(wsp);
    auto take = [&](size_t n) {
        char* r = q;
        q += (n + 255) / 256 * 256;
        return r;
    };
    CgScalars* d_st = reinterpret_cast<CgScalars*>(take(sizeof(CgScalars) * nseg));
    BSeg* d_seg = reinterpret_cast<BSeg*>(take(sizeof(BSeg) * nseg));
    HopArgs* d_args = reinterpret_cast<HopArgs*>(take(sizeof(HopArgs) * nhopk * nlat));
    int* d_off = reinterpret_cast<int*>(take(sizeof(int) * 2 * (nlat + 1)));
    double* d_part = reinterpret_cast<double*>(take(sizeof(double) * npart));
    double* d_red = reinterpret_cast<double*>(take(sizeof(double) * 2 * nseg));
    unsigned* d_tick = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * nseg));
    std::vector<CgScalars> host_st(nseg);
    std::vector<double> hred(2 * nseg);
    if (cudaMemsetAsync(d_tick, 0, sizeof(unsigned) * nseg, s) != cudaSuccess) return LQ_ERR_CUDA;

    // launch descriptors of every lattice for the 2 or 4 hops of K^dag K (p -> q)
    std::vector<HopArgs> args(nhopk * nlat);
    std::vector<int> off1(nlat + 1, 0), off2(nlat + 1, 0);  // work-item prefix sums: one parity / two parities
    for (int l = 0; l < nlat; ++l) {
        Lat& L = lat[l];
        lq_handle* h = L.h;
        h->skip = &d_st[l * nr].done;
        h->skip_stride = (int)(sizeof(CgScalars) / sizeof(int));
        HopArgs* a = &args[l];
        if (op == LQ_OP_WILSON_NORMAL) {
            rc = prep_wilson_full(h, ip, L.t, L.p, nr, &a[0 * nlat], s);
            if (!rc) rc = prep_wilson_full(h, ip, L.q, L.t, nr, &a[1 * nlat], s);
        } else {
            rc = prep_wilson_block(h, ip, L.tmp, L.p, 1, nr, 1.0, &a[0 * nlat], s);
            if (!rc) rc = prep_wilson_schur2(h, ip, L.t, L.tmp, L.p, nr, &a[1 * nlat], s);
            if (!rc) rc = prep_wilson_block(h, ip, L.tmp2, L.t, 1, nr, 1.0, &a[2 * nlat], s);
            if (!rc) rc = prep_wilson_schur2(h, ip, L.q, L.tmp2, L.t, nr, &a[3 * nlat], s);
        }
        h->skip = nullptr;
        if (rc) return rc;
    }

    // autotuning of the persistent hop: sites per work item (x 128) of each lattice and resident blocks
    int occ = 0;
    if (launch_hop_batch(ip, d_args, d_off, nlat, r12, false, op == LQ_OP_WILSON_NORMAL ? EPI_DIAG : EPI_HOP, 0, s,
                         &occ) != cudaSuccess)
        return LQ_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h0->device);
    occ = std::max(occ, 1);
    // the key names the device model (a cached choice is not carried to other GPUs through
    // the cache file) and the batch shape
    char devname[64] = "unknown";
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, h0->device) == cudaSuccess) {
            snprintf(devname, sizeof(devname), "%.63s", prop.name);
            for (char* c = devname; *c; ++c)
                if (*c == ' ' || *c == ':') *c = '_';
        } else {
            cudaGetLastError();
        }
    }
    char keybuf[512];
    int kn = snprintf(keybuf, sizeof(keybuf), "batch:%s:sm%d:p%d:r%d:op%d:n%d", devname, sms, ip, (int)r12, op, nr);
    for (int l = 0; l < nlat && kn < 480; ++l)
        kn += snprintf(keybuf + kn, sizeof(keybuf) - kn, ":%dx%dx%dx%d", hs[l]->g.L[0], hs[l]->g.L[1], hs[l]->g.L[2],
                       hs[l]->g.L[3]);
    const std::string key(keybuf);
    // work-item offsets and the lattices' tile sizes in the launch descriptors, for a shape
    auto shape_for = [&](const Tune& tu) -> int {
        for (int l = 0; l < nlat; ++l) {
            const int m = tu.mult[l];
            const int tiles = (hs[l]->g.Vh + kHopThreads * m - 1) / (kHopThreads * m);
            off1[l + 1] = off1[l] + tiles * nr;
            off2[l + 1] = off2[l] + tiles * nr * 2;
            for (int k = 0; k < nhopk; ++k) args[k * nlat + l].batch_mult = m;
        }
        std::vector<int> both(off1);
        both.insert(both.end(), off2.begin(), off2.end());
        return cudaMemcpyAsync(d_off, both.data(), sizeof(int) * both.size(), cudaMemcpyHostToDevice, s) ==
                               cudaSuccess &&
                       cudaMemcpyAsync(d_args, args.data(), sizeof(HopArgs) * args.size(), cudaMemcpyHostToDevice,
                                       s) == cudaSuccess
                   ? LQ_OK
                   : LQ_ERR_CUDA;
    };
    auto op_launches = [&](const Tune& tu) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < nhopk && e == cudaSuccess; ++k) {
            const bool full = op == LQ_OP_WILSON_NORMAL;
            const int epi = full ? EPI_DIAG : ((k & 1) ? EPI_DIAG : EPI_HOP);
            const bool dag = full ? (k == 1) : (k >= 2);
            e = launch_hop_batch(ip, d_args + k * nlat, full ? d_off + (nlat + 1) : d_off, nlat, r12, dag, epi,
                                 tu.grid, s, nullptr);
        }
        return e;
    };
    Tune best{std::vector<int>(nlat, 1), sms * occ};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_file_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end() && (int)it->second.mult.size() == nlat) {
            best = it->second;
        } else {
            // the operator reads p: give it a defined value (zero) for the timing runs
            for (auto& L : lat)
                if (cudaMemsetAsync(L.p, 0, L.bp, s) != cudaSuccess) return LQ_ERR_CUDA;
            if (cudaMemsetAsync(d_st, 0, sizeof(CgScalars) * nseg, s) != cudaSuccess) return LQ_ERR_CUDA;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            auto time_of = [&](const Tune& c, float* ms) -> int {
                int r = shape_for(c);
                if (r) return r;
                if (op_launches(c) != cudaSuccess) return LQ_ERR_CUDA;  // warm-up
                cudaEventRecord(e0, s);
                for (int k = 0; k < 3; ++k) op_launches(c);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) return LQ_ERR_CUDA;
                cudaEventElapsedTime(ms, e0, e1);
                return LQ_OK;
            };
            // coordinate descent: each lattice's tile size (1, 2, 4 or 8 tiles of 128 sites per item)
            // with the others held, smallest lattice first, at one wave of resident blocks; then the
            // grid (one, two or four waves) for the chosen sizes
            float best_ms = 1e30f;
            rc = time_of(best, &best_ms);
            for (int l = 0; l < nlat && !rc; ++l) {
                for (int m : {2, 4, 8}) {
                    if (kHopThreads * m > 2 * hs[l]->g.Vh) break;  // a single item would exceed the lattice
                    Tune c = best;
                    c.mult[l] = m;
                    float ms = 0;
                    if ((rc = time_of(c, &ms))) break;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
            }
            for (int w : {2, 4}) {
                if (rc) break;
                Tune c = best;
                c.grid = sms * occ * w;
                float ms = 0;
                if ((rc = time_of(c, &ms))) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc) return rc;
            g_tune[key] = best;
            tune_file_save();
        }
    }
    if ((rc = shape_for(best))) return rc;

    // segment table for the vector steps
    std::vector<BSeg> seg(nseg);
    for (int l = 0; l < nlat; ++l) {
        Lat& L = lat[l];
        const size_t sx = L.b32 / nr, sp = L.bp / nr;
        for (int k = 0; k < nr; ++k) {
            BSeg& g = seg[l * nr + k];
            g.x = L.E + k * sx;
            g.r = L.r + k * sx;
            g.p = L.p + k * sp;
            g.q = L.q + k * sp;
            g.Vh = L.h->g.Vh;
            g.nblk = L.nblk;
            g.st = d_st + l * nr + k;
            g.partial = d_part + (size_t)(l * nr + k) * gx;
            g.ticket = d_tick + l * nr + k;
        }
    }
    if (cudaMemcpyAsync(d_seg, seg.data(), sizeof(BSeg) * nseg, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return LQ_ERR_CUDA;

    // the inner iteration, captured once: operator (2 or 4 persistent launches), alpha, update, xpay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LQ_ERR_CUDA;
    cudaError_t ce = cudaSuccess;
    for (int it = 0; it < kIters && ce == cudaSuccess; ++it) {
        ce = op_launches(best);
        if (ce == cudaSuccess) ce = launch_bdot_alpha(d_seg, nseg, gx, ip, s);
        if (ce == cudaSuccess) ce = launch_bupdate(d_seg, nseg, gx, LQ_F32, ip, s);
        if (ce == cudaSuccess) ce = launch_bxpay(d_seg, nseg, gx, ip, LQ_F32, s);
    }
    cudaError_t ce2 = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess || ce2 != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return LQ_ERR_CUDA;
    }
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    };

    // user fields -> native working precision
    for (int l = 0; l < nlat; ++l) {
        Lat& L = lat[l];
        const bool full = L.subset == LQ_FULL;
        char* bw = mixed ? L.B64 : L.RIN;
        cudaError_t e = native ? launch_native_convert(wp, bw, fprec, bs[l], L.h->g.Vh, L.nblk * nr, s)
                               : launch_spinor_to_native(wp, bw, fprec, bs[l], L.h->g, full, 0, nr, s);
        if (e != cudaSuccess) {
            cleanup();
            return LQ_ERR_CUDA;
        }
    }
    std::vector<int> iters(nseg, 0), status(nseg, LQ_OK), outer(nseg, 0);
    std::vector<double> rel(nseg, 0.0), bb(nseg, 0.0);
    std::vector<char> conv(nseg, 0), brk(nseg, 0);  // brk: an inner CG broke down at its first step
    Scratch sc{d_part, d_tick};
    auto norms = [&](int l, char* v, int prec, double* out) -> int {
        Lat& L = lat[l];
        VecRef vr{v, prec, (size_t)L.nblk * spinor_site_bytes(prec) * L.h->g.Vh};
        if (launch_dot(vr, vr, L.h->g.Vh, L.nblk, nr, sc, nullptr, d_red, FIN_STORE, s) != cudaSuccess ||
            cudaMemcpyAsync(hred.data(), d_red, sizeof(double) * nr, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LQ_ERR_CUDA;
        for (int k = 0; k < nr; ++k) out[k] = hred[k];
        return LQ_OK;
    };
    // inner solve: e = 0, r = rhs (FP32), p = r; run the graph until every segment is done
    auto inner = [&](double itol, int maxit) -> int {
        for (int l = 0; l < nlat; ++l) {
            Lat& L = lat[l];
            const size_t strideP = (size_t)L.nblk * spinor_site_bytes(ip) * L.h->g.Vh;
            const size_t stride32 = (size_t)L.nblk * spinor_site_bytes(LQ_F32) * L.h->g.Vh;
            VecRef p{L.p, ip, strideP}, r{L.r, LQ_F32, stride32}, rin{L.RIN, LQ_F32, stride32};
            if (cudaMemsetAsync(L.E, 0, L.b32, s) != cudaSuccess ||
                cudaMemcpyAsync(L.r, L.RIN, L.b32, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                launch_axpby(p, r, 1.0, 0.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess ||
                launch_dot(rin, rin, L.h->g.Vh, L.nblk, nr, sc, nullptr, d_red, FIN_STORE, s) != cudaSuccess ||
                launch_cg_init(d_st + l * nr, d_red, d_red, itol, maxit, nr, s) != cudaSuccess)
                return LQ_ERR_CUDA;
        }
        const int max_launches = maxit / kIters + 2;
        for (int it = 0; it < max_launches; ++it) {
            if (cudaGraphLaunch(exec, s) != cudaSuccess ||
                cudaMemcpyAsync(host_st.data(), d_st, sizeof(CgScalars) * nseg, cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return LQ_ERR_CUDA;
            bool all = true;
            for (int g = 0; g < nseg; ++g) all = all && host_st[g].done;
            if (all) break;
        }
        return LQ_OK;
    };

    // FP32 middle level: e = sum of inner corrections with A e = RIN to `target` (relative, per
    // segment); the FP32 residual RIN0 - A e of every lattice is formed with its own FP32 operator.
    // On return E holds e (the outer loop adds it to the FP64 solution).
    auto middle = [&](double target, double itol, int maxit, std::vector<int>& its, int* most_out) -> int {
        std::vector<double> r0(nseg, 0.0), rn(nseg, 0.0), relm(nseg, 1.0);
        for (int l = 0; l < nlat; ++l) {
            Lat& L = lat[l];
            if (cudaMemcpyAsync(L.RIN0, L.RIN, L.b32, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemsetAsync(L.EM, 0, L.b32, s) != cudaSuccess)
                return LQ_ERR_CUDA;
            int e = norms(l, L.RIN0, LQ_F32, &r0[l * nr]);
            if (e) return e;
        }
        int used = 0, most = 0;
        for (int pass = 0; pass < 8 && used < maxit; ++pass) {
            double reach = 0.5;
            for (int g = 0; g < nseg; ++g)
                if (r0[g] > 0 && relm[g] > target) reach = std::min(reach, 0.5 * target / relm[g]);
            int e = inner(std::max(itol, reach), maxit - used);
            if (e) return e;
            int m = 0;
            for (int g = 0; g < nseg; ++g) {
                its[g] += host_st[g].iter;
                m = std::max(m, host_st[g].iter);
                if (r0[g] > 0 && host_st[g].status == LQ_ERR_BREAKDOWN && host_st[g].iter == 0) brk[g] = 1;
            }
            used += std::max(m, 1);
            most += m;
            bool done = true;
            for (int l = 0; l < nlat; ++l) {
                Lat& L = lat[l];
                const size_t s32 = (size_t)L.nblk * spinor_site_bytes(LQ_F32) * L.h->g.Vh;
                VecRef EMv{L.EM, LQ_F32, s32}, Ev{L.E, LQ_F32, s32}, R0{L.RIN0, LQ_F32, s32},
                    Rv{L.RIN, LQ_F32, s32}, Q{L.q32, LQ_F32, s32};
                if (launch_axpby(EMv, Ev, 1.0, 1.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess) return LQ_ERR_CUDA;
                if ((e = apply_normal_one(L, op, LQ_F32, L.q32, L.EM, L.t32, L.tmp32, nr, s))) return e;
                if (launch_axpby(Rv, R0, 1.0, 0.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess ||
                    launch_axpby(Rv, Q, -1.0, 1.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess)
                    return LQ_ERR_CUDA;
                if ((e = norms(l, L.RIN, LQ_F32, &rn[l * nr]))) return e;
                for (int k = 0; k < nr; ++k) {
                    const int g = l * nr + k;
                    if (r0[g] > 0) its[g] += 1;  // the FP32 residual is one more operator application
                    relm[g] = r0[g] > 0 ? std::sqrt(rn[k + l * nr] / r0[g]) : 0.0;
                    done = done && relm[g] <= target;
                }
            }
            if (done) break;
        }
        for (int l = 0; l < nlat; ++l)
            if (cudaMemcpyAsync(lat[l].E, lat[l].EM, lat[l].b32, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return LQ_ERR_CUDA;
        *most_out = most;
        return LQ_OK;
    };

    if (!mixed) {
        // plain FP32 CG: b is RIN, the solution accumulates in E
        if ((rc = inner(cp->tol, cp->maxiter))) {
            cleanup();
            return rc;
        }
        for (int g = 0; g < nseg; ++g) {
            iters[g] = host_st[g].iter;
            status[g] = host_st[g].status;
            rel[g] = host_st[g].bb > 0 ? std::sqrt(host_st[g].rr / host_st[g].bb) : 0.0;
        }
    } else {
        for (int l = 0; l < nlat; ++l) {
            if (cp->x0_is_guess) {
                Lat& L = lat[l];
                const bool full = L.subset == LQ_FULL;
                cudaError_t e = native ? launch_native_convert(LQ_F64, L.X64, fprec, xs[l], L.h->g.Vh, L.nblk * nr, s)
                                       : launch_spinor_to_native(LQ_F64, L.X64, fprec, xs[l], L.h->g, full, 0, nr, s);
                if (e != cudaSuccess) {
                    cleanup();
                    return LQ_ERR_CUDA;
                }
            } else if (cudaMemsetAsync(lat[l].X64, 0, lat[l].b64, s) != cudaSuccess) {
                cleanup();
                return LQ_ERR_CUDA;
            }
            if ((rc = norms(l, lat[l].B64, LQ_F64, &bb[l * nr]))) {
                cleanup();
                return rc;
            }
        }
        const double itol = cp->inner_tol > 0 ? cp->inner_tol : (ip == LQ_F32 ? 1e-6 : ip == LQ_F16 ? 1e-3 : 3e-2);
        std::vector<double> best_rel(nseg, 1e300);
        std::vector<int> stall(nseg, 0);
        int total_inner = 0;
        bool first = !cp->x0_is_guess;
        for (;;) {
            for (int l = 0; l < nlat && rc == LQ_OK; ++l) {
                Lat& L = lat[l];
                const size_t s64 = (size_t)L.nblk * spinor_site_bytes(LQ_F64) * L.h->g.Vh;
                VecRef R{L.R64, LQ_F64, s64}, B{L.B64, LQ_F64, s64}, Q{L.q64, LQ_F64, s64};
                if (first) {
                    if (launch_axpby(R, B, 1.0, 0.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess) rc = LQ_ERR_CUDA;
                } else {
                    rc = apply_normal_one(L, op, LQ_F64, L.q64, L.X64, L.t64, L.tmp64, nr, s);
                    if (!rc && (launch_axpby(R, B, 1.0, 0.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess ||
                                launch_axpby(R, Q, -1.0, 1.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess))
                        rc = LQ_ERR_CUDA;
                    for (int k = 0; k < nr; ++k) iters[l * nr + k] += conv[l * nr + k] ? 0 : 1;
                }
                std::vector<double> rr(nr);
                if (!rc) rc = norms(l, L.R64, LQ_F64, rr.data());
                for (int k = 0; k < nr && !rc; ++k) {
                    const int g = l * nr + k;
                    rel[g] = bb[g] > 0 ? std::sqrt(rr[k] / bb[g]) : std::sqrt(rr[k]);
                    if (!std::isfinite(rel[g])) status[g] = LQ_ERR_NAN;
                    if (rel[g] < 0.5 * best_rel[g]) {
                        best_rel[g] = rel[g];
                        stall[g] = 0;
                    } else if (++stall[g] >= 3 && rel[g] >= cp->tol) {
                        status[g] = LQ_ERR_NOT_CONVERGED;
                    }
                    conv[g] = conv[g] || rel[g] < cp->tol || status[g] != LQ_OK;
                }
            }
            first = false;
            if (rc) break;
            bool all = true;
            for (int g = 0; g < nseg; ++g) all = all && conv[g];
            if (all) break;
            if (total_inner >= cp->maxiter) {
                for (int g = 0; g < nseg; ++g)
                    if (!conv[g]) status[g] = LQ_ERR_NOT_CONVERGED;
                break;
            }
            for (int l = 0; l < nlat && rc == LQ_OK; ++l) {
                Lat& L = lat[l];
                const size_t s64 = (size_t)L.nblk * spinor_site_bytes(LQ_F64) * L.h->g.Vh;
                const size_t s32 = (size_t)L.nblk * spinor_site_bytes(LQ_F32) * L.h->g.Vh;
                VecRef RIN{L.RIN, LQ_F32, s32}, R{L.R64, LQ_F64, s64};
                if (launch_axpby(RIN, R, 1.0, 0.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess) rc = LQ_ERR_CUDA;
                for (int k = 0; k < nr && !rc; ++k)
                    if (conv[l * nr + k] && cudaMemsetAsync(L.RIN + k * s32, 0, s32, s) != cudaSuccess)
                        rc = LQ_ERR_CUDA;
            }
            // inner tolerance: the precision's floor, or less work once the outer target is within reach
            double reach = 0.5;  // the smallest reduction every unfinished right-hand side still needs
            for (int g = 0; g < nseg; ++g)
                if (!conv[g] && rel[g] > 0) reach = std::min(reach, 0.5 * cp->tol / rel[g]);
            int most = 0;
            if (ip == LQ_F32) {
                const double need = std::max(itol, reach);
                if (rc || (rc = inner(need, cp->maxiter - total_inner))) break;
                for (int g = 0; g < nseg; ++g) {
                    iters[g] += host_st[g].iter;
                    most = std::max(most, host_st[g].iter);
                    // <p, A p> not positive at the first step, with p = r != 0: A is singular on r
                    if (!conv[g] && host_st[g].status == LQ_ERR_BREAKDOWN && host_st[g].iter == 0)
                        status[g] = LQ_ERR_BREAKDOWN;
                }
            } else {
                // three precisions, as in cg.cu: an FP32 defect correction (FP32 residuals of every
                // lattice) around the batched 16-bit inner CG takes each correction to FP32's reach,
                // so the FP64 residuals above are needed about twice per solve
                if (rc || (rc = middle(std::max(kMiddleTolBatch, reach), itol, cp->maxiter - total_inner,
                                       iters, &most)))
                    break;
                for (int g = 0; g < nseg; ++g)
                    if (!conv[g] && brk[g]) status[g] = LQ_ERR_BREAKDOWN;
            }
            for (int g = 0; g < nseg; ++g)
                if (!conv[g]) outer[g] += 1;
            total_inner += std::max(most, 1);
            for (int l = 0; l < nlat && rc == LQ_OK; ++l) {
                Lat& L = lat[l];
                const size_t s64 = (size_t)L.nblk * spinor_site_bytes(LQ_F64) * L.h->g.Vh;
                const size_t s32 = (size_t)L.nblk * spinor_site_bytes(LQ_F32) * L.h->g.Vh;
                VecRef X{L.X64, LQ_F64, s64}, E{L.E, LQ_F32, s32};
                if (launch_axpby(X, E, 1.0, 1.0, L.h->g.Vh, L.nblk, nr, s) != cudaSuccess) rc = LQ_ERR_CUDA;
            }
            if (rc) break;
        }
    }
    cleanup();
    if (rc) return rc;
    // native working precision -> user layout
    for (int l = 0; l < nlat; ++l) {
        Lat& L = lat[l];
        const bool full = L.subset == LQ_FULL;
        char* xw = mixed ? L.X64 : L.E;
        cudaError_t e = native ? launch_native_convert(fprec, xs[l], wp, xw, L.h->g.Vh, L.nblk * nr, s)
                               : launch_spinor_from_native(fprec, xs[l], wp, xw, L.h->g, full, 0, nr, s);
        if (e != cudaSuccess) return LQ_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return LQ_ERR_CUDA;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int ret = LQ_OK;
    for (int g = 0; g < nseg; ++g) {
        stats[g].iters = iters[g];
        stats[g].outer_iters = outer[g];
        stats[g].status = status[g];
        stats[g].true_rel_residual = rel[g];
        stats[g].time_ms = ms;
        if (status[g] != LQ_OK && ret == LQ_OK) ret = status[g];
    }
    return ret;
}
