// blas.cu -- vector kernels for the solvers: the CG updates with their FP64
// global reductions fused in, generic axpby / norms, and the device-side CG
// scalar arithmetic.  Reductions: per-thread FP64 partial sums, warp shuffles,
// a shared-memory block reduction, one partial per block in scratch, and the
// last block to finish (atomic ticket) sums the partials in a fixed order and
// finalises the CG scalars on the device -- no host round trip per iteration.
#include "blas.h"

#include <algorithm>

#include "pdl.cuh"

namespace lq {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce v; thread 0 writes the partial, and the last block of this rhs
// returns true in every thread with `total` set (fixed-order sum of partials).
__device__ bool reduce_last(double v, double* partial, unsigned* ticket, int nblk_x, double& total) {
    __shared__ double ws[kThreads / 32];
    __shared__ bool last;
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        partial[blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == (unsigned)nblk_x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0;
    for (int b = threadIdx.x; b < nblk_x; b += blockDim.x) s += __ldcg(partial + b);
    // deterministic: fixed thread -> partial assignment, then a fixed-shape tree
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) ws[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        total = t;
        *ticket = 0;  // ready for the next launch
    }
    __syncthreads();
    return true;
}

template <int P, typename T>
__device__ __forceinline__ const char* blk_ptr(const VecRef& v, int rhs, int b, int Vh) {
    return v.ptr + (size_t)rhs * v.rhs_stride + (size_t)b * spinor_site_bytes(P) * Vh;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Arithmetic type of a vector kernel: FP64 if any operand is stored in FP64, else FP32.
template <int... Ps>
struct ComputeT {
    static constexpr int prec = ((Ps == LQ_F64) || ...) ? LQ_F64 : LQ_F32;
    using type = typename std::conditional<prec == LQ_F64, double, float>::type;
};
template <int... Ps>
using Compute = typename ComputeT<Ps...>::type;

// ---------------------------------------------------------------- kernels

// sum_re <a, b> per rhs; finalize: FIN_ALPHA (pAp -> alpha) or store into out[rhs]
template <int PA, int PB>
__global__ void __launch_bounds__(kThreads) dot_kernel(VecRef a, VecRef b, int Vh, int nblk, double* scratch,
                                                       unsigned* tickets, CgScalars* st, double* out, int fin) {
    pdl_enter();
    const int rhs = blockIdx.y;
    if (st && st[rhs].done) return;
    using T = Compute<PA, PB>;
    double acc = 0;
    const long n = (long)Vh * nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / Vh), i = (int)(j - (long)bk * Vh);
        cplx<T> sa[12], sb[12];
        load_spinor<PA, T>(blk_ptr<PA, T>(a, rhs, bk, Vh), Vh, i, sa);
        load_spinor<PB, T>(blk_ptr<PB, T>(b, rhs, bk, Vh), Vh, i, sb);
        T site = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) site += sa[k].re * sb[k].re + sa[k].im * sb[k].im;
        acc += (double)site;
    }
    double total;
    if (!reduce_last(acc, scratch + (size_t)rhs * gridDim.x, tickets + rhs, gridDim.x, total)) return;
    if (threadIdx.x != 0) return;
    if (fin == FIN_ALPHA) {
        CgScalars& s = st[rhs];
        s.pAp = total;
        if (!(total > 0.0) || !finite(total)) {
            s.done = 1;
            s.status = LQ_ERR_BREAKDOWN;
            s.alpha = 0;
        } else {
            s.alpha = s.rr / total;
        }
    } else if (out) {
        out[rhs] = total;
    }
}

// x += alpha p ; r -= alpha q ; rr_new = |r|^2 ; beta, convergence (per rhs)
template <int PX, int PP, int PR, int PQ>
__global__ void __launch_bounds__(kThreads) cg_update_kernel(VecRef x, VecRef p, VecRef r, VecRef q, int Vh, int nblk,
                                                             double* scratch, unsigned* tickets, CgScalars* st) {
    pdl_enter();
    const int rhs = blockIdx.y;
    CgScalars& s = st[rhs];
    if (s.done) return;
    using T = Compute<PX, PP, PR, PQ>;
    const T alpha = (T)s.alpha;
    double acc = 0;
    const long n = (long)Vh * nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / Vh), i = (int)(j - (long)bk * Vh);
        cplx<T> xs[12], ps[12], rs[12], qs[12];
        load_spinor<PX, T>(blk_ptr<PX, T>(x, rhs, bk, Vh), Vh, i, xs);
        load_spinor<PP, T>(blk_ptr<PP, T>(p, rhs, bk, Vh), Vh, i, ps);
        load_spinor<PR, T>(blk_ptr<PR, T>(r, rhs, bk, Vh), Vh, i, rs);
        load_spinor<PQ, T>(blk_ptr<PQ, T>(q, rhs, bk, Vh), Vh, i, qs);
        T site = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xs[k].re = fma(alpha, ps[k].re, xs[k].re);
            xs[k].im = fma(alpha, ps[k].im, xs[k].im);
            rs[k].re = fma(-alpha, qs[k].re, rs[k].re);
            rs[k].im = fma(-alpha, qs[k].im, rs[k].im);
            site += rs[k].re * rs[k].re + rs[k].im * rs[k].im;
        }
        acc += (double)site;
        store_spinor<PX, T>(const_cast<char*>(blk_ptr<PX, T>(x, rhs, bk, Vh)), Vh, i, xs);
        store_spinor<PR, T>(const_cast<char*>(blk_ptr<PR, T>(r, rhs, bk, Vh)), Vh, i, rs);
    }
    double total;
    if (!reduce_last(acc, scratch + (size_t)rhs * gridDim.x, tickets + rhs, gridDim.x, total)) return;
    if (threadIdx.x != 0) return;
    s.iter += 1;
    if (!finite(total)) {
        s.done = 1;
        s.status = LQ_ERR_NAN;
        return;
    }
    s.beta = total / s.rr;
    s.rr = total;
    if (total <= s.stop2) s.done = 1;
    else if (s.iter >= s.maxiter) {
        s.done = 1;
        s.status = LQ_ERR_NOT_CONVERGED;
    }
}

// p = r + beta p
template <int PP, int PR>
__global__ void __launch_bounds__(kThreads) cg_xpay_kernel(VecRef p, VecRef r, int Vh, int nblk, const CgScalars* st) {
    pdl_enter();
    const int rhs = blockIdx.y;
    if (st[rhs].done) return;
    using T = Compute<PP, PR>;
    const T beta = (T)st[rhs].beta;
    const long n = (long)Vh * nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / Vh), i = (int)(j - (long)bk * Vh);
        cplx<T> ps[12], rs[12];
        load_spinor<PP, T>(blk_ptr<PP, T>(p, rhs, bk, Vh), Vh, i, ps);
        load_spinor<PR, T>(blk_ptr<PR, T>(r, rhs, bk, Vh), Vh, i, rs);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ps[k].re = fma(beta, ps[k].re, rs[k].re);
            ps[k].im = fma(beta, ps[k].im, rs[k].im);
        }
        store_spinor<PP, T>(const_cast<char*>(blk_ptr<PP, T>(p, rhs, bk, Vh)), Vh, i, ps);
    }
}

// y = a x + b y with host scalars (a applies to every rhs).  The arithmetic is
// that of the output: FP64 for an FP64 y, else FP32 (an FP64 x is rounded to
// FP32 on load; the stored result carries FP32 precision either way, and FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU).
template <int PY, int PX>
__global__ void __launch_bounds__(kThreads) axpby_kernel(VecRef y, VecRef x, double ca_d, double cb_d, int Vh,
                                                         int nblk) {
    pdl_enter();
    using T = typename std::conditional<PY == LQ_F64, double, float>::type;
    const T ca = (T)ca_d, cb = (T)cb_d;
    const int rhs = blockIdx.y;
    const long n = (long)Vh * nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / Vh), i = (int)(j - (long)bk * Vh);
        cplx<T> ys[12], xs[12];
        load_spinor<PX, T>(blk_ptr<PX, T>(x, rhs, bk, Vh), Vh, i, xs);
        if (cb_d != 0.0) load_spinor<PY, T>(blk_ptr<PY, T>(y, rhs, bk, Vh), Vh, i, ys);
        else {
#pragma unroll
            for (int k = 0; k < 12; ++k) ys[k] = {(T)0, (T)0};
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ys[k].re = ca * xs[k].re + cb * ys[k].re;
            ys[k].im = ca * xs[k].im + cb * ys[k].im;
        }
        store_spinor<PY, T>(const_cast<char*>(blk_ptr<PY, T>(y, rhs, bk, Vh)), Vh, i, ys);
    }
}

// CG start: rr = |r|^2 per rhs (already in out), set the scalars
__global__ void cg_init_kernel(CgScalars* st, const double* rr, const double* bb, double tol, int maxiter, int nrhs) {
    pdl_enter();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    CgScalars& s = st[k];
    s.rr = rr[k];
    s.bb = bb[k];
    s.stop2 = tol * tol * bb[k];
    s.iter = 0;
    s.maxiter = maxiter;
    s.status = LQ_OK;
    s.alpha = s.beta = s.pAp = 0;
    s.done = (rr[k] <= s.stop2) ? 1 : 0;
    if (!isfinite(rr[k])) {
        s.done = 1;
        s.status = LQ_ERR_NAN;
    }
}

// Two-component variant of reduce_last (real and imaginary parts).
__device__ bool reduce_last2(double v0, double v1, double* partial, unsigned* ticket, int nblk_x, double& t0,
                             double& t1) {
    __shared__ double ws[2][kThreads / 32];
    __shared__ bool last;
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        ws[0][wid] = v0;
        ws[1][wid] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += ws[0][w];
            s1 += ws[1][w];
        }
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == (unsigned)nblk_x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s0 = 0, s1 = 0;
    for (int b = threadIdx.x; b < nblk_x; b += blockDim.x) {
        s0 += __ldcg(partial + 2 * b);
        s1 += __ldcg(partial + 2 * b + 1);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    __syncthreads();
    if (lane == 0) {
        ws[0][wid] = s0;
        ws[1][wid] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0, a1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a0 += ws[0][w];
            a1 += ws[1][w];
        }
        t0 = a0;
        t1 = a1;
        *ticket = 0;
    }
    __syncthreads();
    return true;
}

// 12 complex numbers of site j of one right-hand side, native or site-major
template <int P, bool NATIVE>
__device__ __forceinline__ void load_site(const char* base, size_t rhs_stride, int rhs, long j, int Vh,
                                          cplx<double> (&s)[12]) {
    const char* r = base + (size_t)rhs * rhs_stride;
    if constexpr (NATIVE) {
        const int bk = (int)(j / Vh), i = (int)(j - (long)bk * Vh);
        load_spinor<P, double>(r + (size_t)bk * spinor_site_bytes(P) * Vh, Vh, i, s);
    } else if constexpr (P == LQ_F64) {
        const double2* q = reinterpret_cast<const double2*>(r) + j * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = q[k];
            s[k] = {v.x, v.y};
        }
    } else {
        const float2* q = reinterpret_cast<const float2*>(r) + j * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 v = q[k];
            s[k] = {(double)v.x, (double)v.y};
        }
    }
}

// <a, b> = sum conj(a) b per right-hand side, FP64 accumulation; result[2 rhs + {0,1}] = (re, im)
template <int P, bool NATIVE>
__global__ void __launch_bounds__(kThreads) cdot_kernel(const char* a, const char* b, size_t rhs_stride, long nsites,
                                                        int Vh, double* scratch, unsigned* tickets, double* result) {
    pdl_enter();
    const int rhs = blockIdx.y;
    double re = 0, im = 0;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < nsites; j += (long)gridDim.x * blockDim.x) {
        cplx<double> sa[12], sb[12];
        load_site<P, NATIVE>(a, rhs_stride, rhs, j, Vh, sa);
        load_site<P, NATIVE>(b, rhs_stride, rhs, j, Vh, sb);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            re += sa[k].re * sb[k].re + sa[k].im * sb[k].im;
            im += sa[k].re * sb[k].im - sa[k].im * sb[k].re;
        }
    }
    double t0, t1;
    if (!reduce_last2(re, im, scratch + (size_t)rhs * 2 * gridDim.x, tickets + rhs, gridDim.x, t0, t1)) return;
    if (threadIdx.x == 0) {
        result[2 * rhs] = t0;
        result[2 * rhs + 1] = t1;
    }
}

// Sum of a group's warp partials (grid.y = group): each block adds a strided
// share with kFinPer independent loads in flight per thread (the partials were
// just written to L2 by the hop), then the last block to finish sums the block
// partials in a fixed order and sets the CG scalars.
constexpr int kFinThreads = 256, kFinPer = 8;

__global__ void __launch_bounds__(kFinThreads) hop_norm_finalize_kernel(const double* partial, int nwarps,
                                                                          CgScalars* st, double* scratch,
                                                                          unsigned* tickets) {
    pdl_enter();
    const int g = blockIdx.y;
    CgScalars& s = st[g];
    if (s.done) return;
    const double* p = partial + (size_t)g * nwarps;
    const int stride = gridDim.x * kFinThreads;
    double acc[kFinPer] = {};
    int w = blockIdx.x * kFinThreads + threadIdx.x;
    for (; w + (kFinPer - 1) * stride < nwarps; w += kFinPer * stride) {
        double v[kFinPer];
#pragma unroll
        for (int u = 0; u < kFinPer; ++u) v[u] = __ldcg(p + w + u * stride);
#pragma unroll
        for (int u = 0; u < kFinPer; ++u) acc[u] += v[u];
    }
    for (; w < nwarps; w += stride) acc[0] += __ldcg(p + w);
    double t = 0;
#pragma unroll
    for (int u = 0; u < kFinPer; ++u) t += acc[u];
    double tot;
    if (!reduce_last(t, scratch + (size_t)g * gridDim.x, tickets + g, gridDim.x, tot)) return;
    if (threadIdx.x == 0) {
        s.pAp = tot;
        if (!(tot > 0.0) || !isfinite(tot)) {
            s.done = 1;
            s.status = LQ_ERR_BREAKDOWN;
            s.alpha = 0;
        } else {
            s.alpha = s.rr / tot;
        }
    }
}

// ------------------------------------------------------- batched segments

template <int P>
__device__ __forceinline__ const char* seg_blk(const char* base, int b, int Vh) {
    return base + (size_t)b * spinor_site_bytes(P) * Vh;
}

template <int PP>
__global__ void __launch_bounds__(kThreads) bdot_alpha_kernel(const BSeg* __restrict__ segs) {
    pdl_enter();
    const BSeg& sg = segs[blockIdx.y];
    if (sg.st->done) return;
    using T = Compute<PP>;
    double acc = 0;
    const long n = (long)sg.Vh * sg.nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / sg.Vh), i = (int)(j - (long)bk * sg.Vh);
        cplx<T> a[12], b[12];
        load_spinor<PP, T>(seg_blk<PP>(sg.p, bk, sg.Vh), sg.Vh, i, a);
        load_spinor<PP, T>(seg_blk<PP>(sg.q, bk, sg.Vh), sg.Vh, i, b);
        T site = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) site += a[k].re * b[k].re + a[k].im * b[k].im;
        acc += (double)site;
    }
    double total;
    if (!reduce_last(acc, sg.partial, sg.ticket, gridDim.x, total)) return;
    if (threadIdx.x != 0) return;
    CgScalars& s = *sg.st;
    s.pAp = total;
    if (!(total > 0.0) || !finite(total)) {
        s.done = 1;
        s.status = LQ_ERR_BREAKDOWN;
        s.alpha = 0;
    } else {
        s.alpha = s.rr / total;
    }
}

template <int PX, int PP>
__global__ void __launch_bounds__(kThreads) bupdate_kernel(const BSeg* __restrict__ segs) {
    pdl_enter();
    const BSeg& sg = segs[blockIdx.y];
    CgScalars& s = *sg.st;
    if (s.done) return;
    using T = Compute<PX, PP>;
    const T alpha = (T)s.alpha;
    double acc = 0;
    const long n = (long)sg.Vh * sg.nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / sg.Vh), i = (int)(j - (long)bk * sg.Vh);
        cplx<T> xs[12], ps[12], rs[12], qs[12];
        load_spinor<PX, T>(seg_blk<PX>(sg.x, bk, sg.Vh), sg.Vh, i, xs);
        load_spinor<PP, T>(seg_blk<PP>(sg.p, bk, sg.Vh), sg.Vh, i, ps);
        load_spinor<PX, T>(seg_blk<PX>(sg.r, bk, sg.Vh), sg.Vh, i, rs);
        load_spinor<PP, T>(seg_blk<PP>(sg.q, bk, sg.Vh), sg.Vh, i, qs);
        T site = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xs[k].re = fma(alpha, ps[k].re, xs[k].re);
            xs[k].im = fma(alpha, ps[k].im, xs[k].im);
            rs[k].re = fma(-alpha, qs[k].re, rs[k].re);
            rs[k].im = fma(-alpha, qs[k].im, rs[k].im);
            site += rs[k].re * rs[k].re + rs[k].im * rs[k].im;
        }
        acc += (double)site;
        store_spinor<PX, T>(const_cast<char*>(seg_blk<PX>(sg.x, bk, sg.Vh)), sg.Vh, i, xs);
        store_spinor<PX, T>(const_cast<char*>(seg_blk<PX>(sg.r, bk, sg.Vh)), sg.Vh, i, rs);
    }
    double total;
    if (!reduce_last(acc, sg.partial, sg.ticket, gridDim.x, total)) return;
    if (threadIdx.x != 0) return;
    s.iter += 1;
    if (!finite(total)) {
        s.done = 1;
        s.status = LQ_ERR_NAN;
        return;
    }
    s.beta = total / s.rr;
    s.rr = total;
    if (total <= s.stop2) s.done = 1;
    else if (s.iter >= s.maxiter) {
        s.done = 1;
        s.status = LQ_ERR_NOT_CONVERGED;
    }
}

template <int PP, int PR>
__global__ void __launch_bounds__(kThreads) bxpay_kernel(const BSeg* __restrict__ segs) {
    pdl_enter();
    const BSeg& sg = segs[blockIdx.y];
    if (sg.st->done) return;
    using T = Compute<PP, PR>;
    const T beta = (T)sg.st->beta;
    const long n = (long)sg.Vh * sg.nblk;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const int bk = (int)(j / sg.Vh), i = (int)(j - (long)bk * sg.Vh);
        cplx<T> ps[12], rs[12];
        load_spinor<PP, T>(seg_blk<PP>(sg.p, bk, sg.Vh), sg.Vh, i, ps);
        load_spinor<PR, T>(seg_blk<PR>(sg.r, bk, sg.Vh), sg.Vh, i, rs);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ps[k].re = fma(beta, ps[k].re, rs[k].re);
            ps[k].im = fma(beta, ps[k].im, rs[k].im);
        }
        store_spinor<PP, T>(const_cast<char*>(seg_blk<PP>(sg.p, bk, sg.Vh)), sg.Vh, i, ps);
    }
}

int grid_x(int Vh, int nblk) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 132;
    }
    const long n = (long)Vh * nblk;
    long want = (n + kThreads - 1) / kThreads;
    const long cap = (long)sms * 8;
    return (int)(want < cap ? want : cap);
}

}  // namespace

#define LQ_P_SWITCH(pv, NAME, BODY)                               \
    switch (pv) {                                                 \
    case LQ_F64: { constexpr int NAME = LQ_F64; BODY; } break;    \
    case LQ_F32: { constexpr int NAME = LQ_F32; BODY; } break;    \
    case LQ_F16: { constexpr int NAME = LQ_F16; BODY; } break;    \
    default: { constexpr int NAME = LQ_BF16; BODY; } break;       \
    }

cudaError_t launch_hop_norm_finalize(const double* partial, int nwarps, int ngroups, CgScalars* st,
                                     const Scratch& sc, int Vh, int nblk, cudaStream_t s) {
    // blocks per group: one per kFinThreads * kFinPer partials, within the scratch
    // entries per right-hand side that the vector kernels use (grid_x)
    const int want = (nwarps + kFinThreads * kFinPer - 1) / (kFinThreads * kFinPer);
    const int nb = std::max(1, std::min(want, grid_x(Vh, nblk)));
    launch_pdl(hop_norm_finalize_kernel, dim3(nb, ngroups), kFinThreads, 0, s, partial, nwarps, st, sc.partial,
               sc.tickets);
    return cudaGetLastError();
}

size_t reduce_scratch_doubles(int Vh, int nblk, int nrhs) { return (size_t)grid_x(Vh, nblk) * nrhs; }

int cdot_grid(long nsites) {
    const long want = (nsites + kThreads - 1) / kThreads;
    const long cap = (long)kMaxGrid;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_cdot(int fmt, const void* a, const void* b, size_t rhs_stride, long nsites, int Vh, int nrhs,
                        double* scratch, unsigned* tickets, double* result, cudaStream_t s) {
    const int prec = fmt & 0xF;
    const bool native = (fmt & LQ_NATIVE) != 0;
    dim3 grid(cdot_grid(nsites), nrhs);
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    if (native) {
        LQ_P_SWITCH(prec, P, (launch_pdl(cdot_kernel<P, true>, grid, kThreads, 0, s, pa, pb, rhs_stride, nsites, Vh, scratch, tickets, result)))
    } else if (prec == LQ_F64) {
        launch_pdl(cdot_kernel<LQ_F64, false>, grid, kThreads, 0, s, pa, pb, rhs_stride, nsites, Vh, scratch, tickets, result);
    } else {
        launch_pdl(cdot_kernel<LQ_F32, false>, grid, kThreads, 0, s, pa, pb, rhs_stride, nsites, Vh, scratch, tickets, result);
    }
    return cudaGetLastError();
}

cudaError_t launch_dot(const VecRef& a, const VecRef& b, int Vh, int nblk, int nrhs, const Scratch& sc,
                       CgScalars* st, double* out, int fin, cudaStream_t s) {
    dim3 grid(grid_x(Vh, nblk), nrhs);
    LQ_P_SWITCH(a.prec, PA, LQ_P_SWITCH(b.prec, PB,
        (launch_pdl(dot_kernel<PA, PB>, grid, kThreads, 0, s, a, b, Vh, nblk, sc.partial, sc.tickets, st, out, fin))))
    return cudaGetLastError();
}

cudaError_t launch_cg_update(const VecRef& x, const VecRef& p, const VecRef& r, const VecRef& q, int Vh, int nblk,
                             int nrhs, const Scratch& sc, CgScalars* st, cudaStream_t s) {
    dim3 grid(grid_x(Vh, nblk), nrhs);
    // precision combinations used by the solvers: all equal; x, r in FP32 with p, q in FP16/BF16;
    // x in FP32 with r, p, q in FP16/BF16
    if (x.prec == LQ_F64 && p.prec == LQ_F64 && r.prec == LQ_F64 && q.prec == LQ_F64)
        launch_pdl(cg_update_kernel<LQ_F64, LQ_F64, LQ_F64, LQ_F64>, grid, kThreads, 0, s, x, p, r, q, Vh, nblk, sc.partial, sc.tickets, st);
    else if (x.prec == LQ_F32 && r.prec == LQ_F32 && p.prec == q.prec) {
        switch (p.prec) {
        case LQ_F32: launch_pdl(cg_update_kernel<LQ_F32, LQ_F32, LQ_F32, LQ_F32>, grid, kThreads, 0, s, x, p, r, q, Vh, nblk, sc.partial, sc.tickets, st); break;
        case LQ_F16: launch_pdl(cg_update_kernel<LQ_F32, LQ_F16, LQ_F32, LQ_F16>, grid, kThreads, 0, s, x, p, r, q, Vh, nblk, sc.partial, sc.tickets, st); break;
        case LQ_BF16: launch_pdl(cg_update_kernel<LQ_F32, LQ_BF16, LQ_F32, LQ_BF16>, grid, kThreads, 0, s, x, p, r, q, Vh, nblk, sc.partial, sc.tickets, st); break;
        default: return cudaErrorInvalidValue;
        }
    } else if (x.prec == LQ_F32 && r.prec == p.prec && p.prec == q.prec && p.prec == LQ_F16) {
        launch_pdl(cg_update_kernel<LQ_F32, LQ_F16, LQ_F16, LQ_F16>, grid, kThreads, 0, s, x, p, r, q, Vh, nblk, sc.partial, sc.tickets, st);
    } else if (x.prec == LQ_F32 && r.prec == p.prec && p.prec == q.prec && p.prec == LQ_BF16) {
        launch_pdl(cg_update_kernel<LQ_F32, LQ_BF16, LQ_BF16, LQ_BF16>, grid, kThreads, 0, s, x, p, r, q, Vh, nblk, sc.partial, sc.tickets, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cg_xpay(const VecRef& p, const VecRef& r, int Vh, int nblk, int nrhs, const CgScalars* st,
                           cudaStream_t s) {
    dim3 grid(grid_x(Vh, nblk), nrhs);
    LQ_P_SWITCH(p.prec, PP, LQ_P_SWITCH(r.prec, PR,
        (launch_pdl(cg_xpay_kernel<PP, PR>, grid, kThreads, 0, s, p, r, Vh, nblk, st))))
    return cudaGetLastError();
}

cudaError_t launch_axpby(const VecRef& y, const VecRef& x, double a, double b, int Vh, int nblk, int nrhs,
                         cudaStream_t s) {
    dim3 grid(grid_x(Vh, nblk), nrhs);
    LQ_P_SWITCH(y.prec, PY, LQ_P_SWITCH(x.prec, PX,
        (launch_pdl(axpby_kernel<PY, PX>, grid, kThreads, 0, s, y, x, a, b, Vh, nblk))))
    return cudaGetLastError();
}

cudaError_t launch_bdot_alpha(const BSeg* segs, int nseg, int gx, int pp, cudaStream_t s) {
    dim3 grid(gx, nseg);
    LQ_P_SWITCH(pp, PP, (launch_pdl(bdot_alpha_kernel<PP>, grid, kThreads, 0, s, segs)))
    return cudaGetLastError();
}

cudaError_t launch_bupdate(const BSeg* segs, int nseg, int gx, int px, int pp, cudaStream_t s) {
    dim3 grid(gx, nseg);
    if (px != LQ_F32 && px != LQ_F64) return cudaErrorInvalidValue;
    if (px == LQ_F64) {
        if (pp != LQ_F64) return cudaErrorInvalidValue;
        launch_pdl(bupdate_kernel<LQ_F64, LQ_F64>, grid, kThreads, 0, s, segs);
    } else {
        switch (pp) {
        case LQ_F32: launch_pdl(bupdate_kernel<LQ_F32, LQ_F32>, grid, kThreads, 0, s, segs); break;
        case LQ_F16: launch_pdl(bupdate_kernel<LQ_F32, LQ_F16>, grid, kThreads, 0, s, segs); break;
        case LQ_BF16: launch_pdl(bupdate_kernel<LQ_F32, LQ_BF16>, grid, kThreads, 0, s, segs); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_bxpay(const BSeg* segs, int nseg, int gx, int pp, int pr, cudaStream_t s) {
    dim3 grid(gx, nseg);
    LQ_P_SWITCH(pp, PP, LQ_P_SWITCH(pr, PR, (launch_pdl(bxpay_kernel<PP, PR>, grid, kThreads, 0, s, segs))))
    return cudaGetLastError();
}

cudaError_t launch_cg_init(CgScalars* st, const double* rr, const double* bb, double tol, int maxiter, int nrhs,
                           cudaStream_t s) {
    launch_pdl(cg_init_kernel, (nrhs + 63) / 64, 64, 0, s, st, rr, bb, tol, maxiter, nrhs);
    return cudaGetLastError();
}

}  // namespace lq
