// blockcg.cu -- block conjugate gradient (O'Leary 1980) for N right-hand
// sides that share one operator A = K^dag K.
//
//   R = B - A X,  P = R
//   repeat:  Q = A P                      (one multi-RHS operator launch set)
//            Delta = P^dag Q = (K P)^dag (K P),  rho = R^dag R
//                                                      (N x N, FP64 sums)
//            alpha = Delta^{-1} rho
//            X += P alpha,  R -= Q alpha
//            beta = rho^{-1} (R^dag R)_new,  P = R + P beta

// The block vectors live in FP32 storage (FP32 arithmetic); the N x N Gram
// matrices are summed on the device (FP32 per-thread sums, FP64 lane and
// block reductions in a fixed order) and the N x N algebra (Cholesky
// solves) runs in FP64 on the host.  Every block kernel reads each column
// once per call (tiles of all N columns staged in shared memory); P is
// updated in place.  As a mixed-precision solver
// the block CG is the inner solve of the FP64 defect-correction loop in
// cg.cu: it stops when every column's residual has dropped by the inner
// tolerance, or when Delta stops being numerically positive definite (the
// block has lost rank), and the FP64 outer loop restarts from the true
// residual.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "blas.h"
#include "blockcg.h"
#include "pdl.cuh"
#include "trace.h"

namespace lq {

namespace {

// Block vectors are N columns of FP32 native fields; column j is a contiguous
// array of M float4 (2 complex numbers each) at base + j * stride4 float4s.
// Every block kernel below walks tiles of kTE consecutive float4 of all N
// columns: the CTA stages the tile of each input matrix in shared memory with
// cp.async (one read of every column from memory), then in the update kernels
// warp w < ceil(N/2) works on the output columns w and w + ceil(N/2), lane l
// on the tile elements l and l + 32 (the Gram kernel splits the work by blocks
// of the result instead).  Blocks have a whole number of kTE-thread groups
// (see block_threads).
constexpr int kTE = 64;
constexpr int kGrid = 152 * 4;  // most blocks of the Gram kernel (its partial sums are sized for it)
constexpr int kGramStages = 3;

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    const int n = valid ? 16 : 0;  // 0: zero-fill, nothing read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// s[j * kTE + e] = column j, element e0 + e (zero past M)
__device__ __forceinline__ void stage_tile(float4* s, const float4* __restrict__ base, size_t stride4, long e0,
                                           long M, int N) {
    const int e = threadIdx.x & (kTE - 1);  // blockDim.x is a multiple of kTE
    const bool ok = e0 + e < M;
    const float4* src = base + (ok ? e0 + e : 0);
    for (int j = threadIdx.x / kTE; j < N; j += blockDim.x / kTE)
        cp_async16(s + j * kTE + e, src + (size_t)j * stride4, ok);
}

// the output columns of this warp in the update kernels: c0 = w, c1 = w + ceil(N/2)
struct WarpCols {
    int c0, c1;
    bool has0, has1;
};
__device__ __forceinline__ WarpCols warp_cols_split(int N) {
    const int w = threadIdx.x >> 5, h = (N + 1) / 2;
    WarpCols c;
    c.c0 = w;
    c.c1 = w + h;
    c.has0 = w < h;
    c.has1 = c.has0 && c.c1 < N;
    return c;
}

// acc += conj(a) * b over the two complex numbers of a float4
__device__ __forceinline__ void cdot4(float2& acc, const float4 a, const float4 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.x = fmaf(a.z, b.z, acc.x);
    acc.x = fmaf(a.w, b.w, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
    acc.y = fmaf(a.z, b.w, acc.y);
    acc.y = fmaf(-a.w, b.z, acc.y);
}

// y += c * x for the two complex numbers of a float4 (c complex)
__device__ __forceinline__ void cmac4(float4& y, const float2 c, const float4 x) {
    y.x = fmaf(c.x, x.x, y.x);
    y.x = fmaf(-c.y, x.y, y.x);
    y.y = fmaf(c.x, x.y, y.y);
    y.y = fmaf(c.y, x.x, y.y);
    y.z = fmaf(c.x, x.z, y.z);
    y.z = fmaf(-c.y, x.w, y.z);
    y.w = fmaf(c.x, x.w, y.w);
    y.w = fmaf(c.y, x.z, y.w);
}

// partial[blk][i][j] = sum over the block's tiles of <A_i, A_j> (conj on the
// first), for i <= j (the rest of the Hermitian result is its conjugate; the
// kernel writes zeros there).  The N columns form groups of kGramGroup; warp w
// owns one kGramGroup x kGramGroup block (I, J), I <= J, of the result and
// keeps its complex sums in registers (on a diagonal block I = J only those
// with r <= c).  A pipeline stage holds kGramSub sub-tiles of kTE float4 of
// every column, column j of a sub-tile at row j (no padding: lane l reads
// element l + 32 u, so a warp's 16-byte loads cover consecutive banks).  Per
// float4 a lane loads the 4 + 4 column values of its block (4 when I = J) and
// does 16 (10) complex products of two complex pairs, from immediate offsets
// of one shared address; whether the block is diagonal and whether all its
// columns exist (N a multiple of 4, or not the last group) are resolved once
// per sub-tile by a warp-uniform branch.  kGramStages stages: the copies of
// the next ones are in flight while the current one is multiplied.  Sums in
// FP32 per lane; the reductions over lanes and blocks in FP64, in a fixed
// order.
constexpr int kGramGroup = 4;
constexpr int kGramSub = 2;

__host__ __device__ constexpr int gram_groups(int N) { return (N + kGramGroup - 1) / kGramGroup; }
__host__ __device__ constexpr int gram_blocks(int N) { return gram_groups(N) * (gram_groups(N) + 1) / 2; }
// one warp per result block, rounded up to whole kTE-thread groups (tile staging)
__host__ __device__ constexpr int gram_threads(int N) { return kTE * ((32 * gram_blocks(N) + kTE - 1) / kTE); }
constexpr int kGramMaxThreads = gram_threads(kMaxBlockRhs);

// acc[r][c] += conj(a_r) b_c for one float4 of the sub-tile: a_r at sa[r * kTE]
// (column 4I + r), b_c at sb[c * kTE] (column 4J + c); na, nb: columns of the
// two groups that exist.  DIAG: sb = sa, and only r <= c.  FULL: na = nb = 4.
template <bool DIAG, bool FULL>
__device__ __forceinline__ void gram_accumulate(float2 (&acc)[kGramGroup][kGramGroup], const float4* sa,
                                                const float4* sb, int na, int nb) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a[kGramGroup], b[kGramGroup];
#pragma unroll
    for (int c = 0; c < kGramGroup; ++c) {
        a[c] = (FULL || c < na) ? sa[c * kTE] : z4;
        if (!DIAG) b[c] = (FULL || c < nb) ? sb[c * kTE] : z4;
    }
#pragma unroll
    for (int r = 0; r < kGramGroup; ++r)
#pragma unroll
        for (int c = 0; c < kGramGroup; ++c)
            if (!DIAG || r <= c) cdot4(acc[r][c], a[r], DIAG ? a[c] : b[c]);
}

__global__ void __launch_bounds__(kGramMaxThreads) block_gram_kernel(const float4* __restrict__ A, size_t stride4,
                                                                     long M, int N, double2* partial) {
    pdl_enter();
    extern __shared__ float4 sm[];
    const size_t sub = (size_t)N * kTE, buf = kGramSub * sub;  // float4 per sub-tile, per stage
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ng = gram_groups(N);
    const bool busy = w < gram_blocks(N);
    int I = 0, r = w;  // this warp's block (I, J) of the result
    while (I < ng && r >= ng - I) {  // row I of the upper triangle holds ng - I blocks
        r -= ng - I;
        ++I;
    }
    const int J = I + r;
    const int na = min(kGramGroup, N - kGramGroup * I), nb = min(kGramGroup, N - kGramGroup * J);
    const int mode = (I == J ? 2 : 0) + (na == kGramGroup && nb == kGramGroup ? 1 : 0);
    float2 acc[kGramGroup][kGramGroup];
#pragma unroll
    for (int a = 0; a < kGramGroup; ++a)
#pragma unroll
        for (int b = 0; b < kGramGroup; ++b) acc[a][b] = make_float2(0.f, 0.f);
    const long span = (long)kGramSub * kTE, step = (long)gridDim.x * span;
    auto stage = [&](long e0, int k) {
        if (e0 < M) {
#pragma unroll
            for (int q = 0; q < kGramSub; ++q) stage_tile(sm + k * buf + q * sub, A, stride4, e0 + q * kTE, M, N);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");  // one group per stage (maybe empty)
    };
#pragma unroll
    for (int k = 0; k < kGramStages - 1; ++k) stage((long)blockIdx.x * span + k * step, k);
    int k = 0;
    for (long e0 = (long)blockIdx.x * span; e0 < M; e0 += step) {
        stage(e0 + (kGramStages - 1) * step, (k + kGramStages - 1) % kGramStages);
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kGramStages - 1) : "memory");  // stage e0 has landed
        __syncthreads();
        if (busy) {
#pragma unroll
            for (int q = 0; q < kGramSub; ++q) {
                // elements past M are zero-filled
                const float4* sa = sm + k * buf + q * sub + kGramGroup * I * kTE + lane;
                const float4* sb = sm + k * buf + q * sub + kGramGroup * J * kTE + lane;
#pragma unroll
                for (int u = 0; u < kTE / 32; ++u) {
                    switch (mode) {
                        case 3: gram_accumulate<true, true>(acc, sa + 32 * u, sa + 32 * u, na, nb); break;
                        case 2: gram_accumulate<true, false>(acc, sa + 32 * u, sa + 32 * u, na, nb); break;
                        case 1: gram_accumulate<false, true>(acc, sa + 32 * u, sb + 32 * u, na, nb); break;
                        default: gram_accumulate<false, false>(acc, sa + 32 * u, sb + 32 * u, na, nb); break;
                    }
                }
            }
        }
        __syncthreads();  // stage k is refilled by a later iteration's copies
        k = (k + 1) % kGramStages;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // lane sums -> one FP64 entry per (i, j) in shared memory (zero where no warp sums) -> partial
    double2* red = reinterpret_cast<double2*>(sm);  // [N][N]
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) red[t] = make_double2(0.0, 0.0);
    __syncthreads();
    if (busy) {
#pragma unroll
        for (int a = 0; a < kGramGroup; ++a)
#pragma unroll
            for (int b = 0; b < kGramGroup; ++b) {
                double x = acc[a][b].x, y = acc[a][b].y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                }
                const int i = kGramGroup * I + a, j = kGramGroup * J + b;
                if (lane == 0 && i <= j && i < N && j < N) red[i * N + j] = make_double2(x, y);
            }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) partial[(size_t)blockIdx.x * N * N + t] = red[t];
}

// G = sum over blocks of the partials: one warp per entry, lanes stride over
// the blocks, then a fixed shuffle tree (the same order on every call).
__global__ void gram_final_kernel(const double2* partial, int nblk, int N, double2* G) {
    pdl_enter();
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= N * N) return;
    double x = 0.0, y = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = partial[(size_t)b * N * N + e];
        x += v.x;
        y += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) G[e] = make_double2(x, y);
}

// X_j += sum_k P_k a[k][j],  R_j -= sum_k Q_k a[k][j]   (a: N x N, row-major, complex).
// (A variant that also summed R^dag R of the new R tile in shared memory was
// measured slower than this kernel plus the separate Gram: 706 us against
// 340 + 213 us on half of 24^3 x 48 with 12 columns, its 126 registers halving
// the resident blocks.)
__global__ void __launch_bounds__(32 * ((kMaxBlockRhs + 1) / 2)) block_update_kernel(
    float4* __restrict__ X, const float4* __restrict__ P, float4* __restrict__ R, const float4* __restrict__ Q,
    size_t stride4, long M, int N, const float2* __restrict__ a) {
    pdl_enter();
    extern __shared__ float4 sm[];
    float4* sP = sm;
    float4* sQ = sm + (size_t)N * kTE;
    float2* sa = reinterpret_cast<float2*>(sm + (size_t)2 * N * kTE);
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) sa[e] = a[e];
    const int lane = threadIdx.x & 31;
    const WarpCols wc = warp_cols_split(N);
    const int j0 = wc.c0, j1 = wc.c1;
    const bool has0 = wc.has0, has1 = wc.has1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long e0 = (long)blockIdx.x * kTE; e0 < M; e0 += (long)gridDim.x * kTE) {
        stage_tile(sP, P, stride4, e0, M, N);
        stage_tile(sQ, Q, stride4, e0, M, N);
        float4 x[2][2], r[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long ge = e0 + lane + 32 * u;
            const bool ok = has0 && ge < M;
            x[0][u] = ok ? X[(size_t)j0 * stride4 + ge] : z4;
            r[0][u] = ok ? R[(size_t)j0 * stride4 + ge] : z4;
            x[1][u] = ok && has1 ? X[(size_t)j1 * stride4 + ge] : z4;
            r[1][u] = ok && has1 ? R[(size_t)j1 * stride4 + ge] : z4;
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kMaxBlockRhs; ++k) {
            if (k < N && has0) {
                const float2 c0 = sa[k * N + j0];
                const float2 c1 = has1 ? sa[k * N + j1] : make_float2(0.f, 0.f);
                const float2 m0 = make_float2(-c0.x, -c0.y), m1 = make_float2(-c1.x, -c1.y);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float4 p = sP[k * kTE + lane + 32 * u];
                    const float4 q = sQ[k * kTE + lane + 32 * u];
                    cmac4(x[0][u], c0, p);
                    cmac4(x[1][u], c1, p);
                    cmac4(r[0][u], m0, q);
                    cmac4(r[1][u], m1, q);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long ge = e0 + lane + 32 * u;
            if (has0 && ge < M) {
                X[(size_t)j0 * stride4 + ge] = x[0][u];
                R[(size_t)j0 * stride4 + ge] = r[0][u];
                if (has1) {
                    X[(size_t)j1 * stride4 + ge] = x[1][u];
                    R[(size_t)j1 * stride4 + ge] = r[1][u];
                }
            }
        }
        __syncthreads();
    }
}

// P_j = R_j + sum_k P_k b[k][j], in place: a tile of every column of P is in
// shared memory before any of it is overwritten, and tiles are disjoint.
__global__ void __launch_bounds__(32 * ((kMaxBlockRhs + 1) / 2)) block_pupdate_kernel(
    float4* __restrict__ P, const float4* __restrict__ R, size_t stride4, long M, int N, const float2* __restrict__ b) {
    pdl_enter();
    extern __shared__ float4 sm[];
    const size_t buf = (size_t)N * kTE;  // the P tile of one of the two stages
    float2* sb = reinterpret_cast<float2*>(sm + 2 * buf);
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) sb[e] = b[e];
    const int lane = threadIdx.x & 31;
    const WarpCols wc = warp_cols_split(N);
    const int j0 = wc.c0, j1 = wc.c1;
    const bool has0 = wc.has0, has1 = wc.has1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const long step = (long)gridDim.x * kTE;
    auto stage = [&](long e0, int k) {
        if (e0 < M) stage_tile(sm + k * buf, P, stride4, e0, M, N);
        asm volatile("cp.async.commit_group;\n" ::: "memory");  // one group per tile (maybe empty)
    };
    stage((long)blockIdx.x * kTE, 0);
    int kb = 0;
    for (long e0 = (long)blockIdx.x * kTE; e0 < M; e0 += step, kb ^= 1) {
        // the next tile's copies run while this one is updated (it is this block's own, and
        // written only in a later iteration)
        stage(e0 + step, kb ^ 1);
        const float4* sP = sm + kb * buf;
        float4 y[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long ge = e0 + lane + 32 * u;
            const bool ok = has0 && ge < M;
            y[0][u] = ok ? R[(size_t)j0 * stride4 + ge] : z4;
            y[1][u] = ok && has1 ? R[(size_t)j1 * stride4 + ge] : z4;
        }
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this tile has landed
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kMaxBlockRhs; ++k) {
            if (k < N && has0) {
                const float2 c0 = sb[k * N + j0];
                const float2 c1 = has1 ? sb[k * N + j1] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float4 p = sP[k * kTE + lane + 32 * u];
                    cmac4(y[0][u], c0, p);
                    cmac4(y[1][u], c1, p);
                }
            }
        }
        __syncthreads();  // every warp has read stage kb before the next iteration refills it
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long ge = e0 + lane + 32 * u;
            if (has0 && ge < M) {
                P[(size_t)j0 * stride4 + ge] = y[0][u];
                if (has1) P[(size_t)j1 * stride4 + ge] = y[1][u];
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// grid of a block kernel: every SM gets the same number of resident blocks
// (a partial second wave would leave most SMs idle at the end), at most cap
// (kGrid for the Gram kernel, whose partial sums are sized for it)
template <typename K>
int block_grid(long M, K kern, int threads, size_t smem, long cap = kGrid) {
    const long want = (M + kTE - 1) / kTE;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1, sms = 152;
    const long resident = std::min<long>((long)per_sm * sms, cap);
    return (int)std::min<long>(want, resident);
}

// threads of the block kernels: one warp per pair of columns, rounded up to
// whole kTE-thread groups (the staging loop assigns one tile element per thread)
int block_threads(int N) {
    const int warps = (N + 1) / 2;
    return kTE * ((32 * warps + kTE - 1) / kTE);
}

using cd = std::complex<double>;

// Solve H Z = Y for Hermitian positive definite H (N x N, row-major) by
// Cholesky; Y and Z are N x N.  Returns false if H is not numerically
// positive definite (pivot <= eps * largest diagonal).
bool chol_solve(const std::vector<cd>& H, const std::vector<cd>& Y, std::vector<cd>& Z, int N) {
    std::vector<cd> L(N * N, 0.0);
    double dmax = 0;
    for (int i = 0; i < N; ++i) dmax = std::max(dmax, H[i * N + i].real());
    for (int j = 0; j < N; ++j) {
        double d = H[j * N + j].real();
        for (int k = 0; k < j; ++k) d -= std::norm(L[j * N + k]);
        if (!(d > 1e-13 * dmax)) return false;
        const double ljj = std::sqrt(d);
        L[j * N + j] = ljj;
        for (int i = j + 1; i < N; ++i) {
            cd s = H[i * N + j];
            for (int k = 0; k < j; ++k) s -= L[i * N + k] * std::conj(L[j * N + k]);
            L[i * N + j] = s / ljj;
        }
    }
    Z = Y;
    for (int c = 0; c < N; ++c) {  // forward: L w = y ; back: L^dag z = w
        for (int i = 0; i < N; ++i) {
            cd s = Z[i * N + c];
            for (int k = 0; k < i; ++k) s -= L[i * N + k] * Z[k * N + c];
            Z[i * N + c] = s / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            cd s = Z[i * N + c];
            for (int k = i + 1; k < N; ++k) s -= std::conj(L[k * N + i]) * Z[k * N + c];
            Z[i * N + c] = s / L[i * N + i];
        }
    }
    return true;
}

}  // namespace

int block_cg(const BlockCgOps& ops, char* X, const char* Bv, char* R, char* P, char* Q, size_t stride, long nsites,
             int N, double tol, int maxiter, void* ws, double2* hostbuf, cudaStream_t s, int* iters) {
    lq::TraceRange trace_("lqcd/cg/block");
    if (N < 1 || N > kMaxBlockRhs || stride % 16 != 0 || !ops.kimage) return LQ_ERR_ARG;
    const long M = nsites * (spinor_site_bytes(LQ_F32) / 16);  // float4 per column
    const size_t stride4 = stride / 16;
    const int nthr = block_threads(N);
    const size_t tile = sizeof(float4) * N * kTE, mat = sizeof(float2) * N * N;
    const size_t gtile = sizeof(float4) * N * kTE * kGramSub;  // Gram stage buffer
    const int t_gram = gram_threads(N);
    double2* partial = static_cast<double2*>(ws);
    double2* Gd = partial + (size_t)kGrid * N * N;
    float2* Md = reinterpret_cast<float2*>(Gd + N * N);
    static bool configured = false;  // the Gram of 16 columns takes 96 KB of stage buffers
    if (!configured) {
        const int gb = (int)(kGramStages * sizeof(float4) * kMaxBlockRhs * kTE * kGramSub);
        if (cudaFuncSetAttribute(block_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, gb) != cudaSuccess)
            return LQ_ERR_CUDA;
        configured = true;
    }
    const int g_gram = block_grid(M, block_gram_kernel, t_gram, kGramStages * gtile);
    const size_t s_upd = 2 * tile + mat;  // the P and Q tiles + the N x N matrix
    const size_t s_pup = 2 * tile + mat;  // two stages of the P tile + the N x N matrix
    const int g_upd = block_grid(M, block_update_kernel, nthr, s_upd, 1L << 30);
    const int g_pup = block_grid(M, block_pupdate_kernel, nthr, s_pup, 1L << 30);
    auto f4 = [](const char* q) { return reinterpret_cast<const float4*>(q); };
    auto w4 = [](char* q) { return reinterpret_cast<float4*>(q); };
    // the Gram of K P runs on a second stream beside the operator's K^dag stage
    cudaStream_t s2 = nullptr;
    cudaEvent_t kdone = nullptr;
    struct Release {
        cudaStream_t& s2;
        cudaEvent_t& ev;
        ~Release() {
            if (ev) cudaEventDestroy(ev);
            if (s2) cudaStreamDestroy(s2);
        }
    } release_{s2, kdone};
    if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&kdone, cudaEventDisableTiming) != cudaSuccess)
        return LQ_ERR_CUDA;
    // G = A^dag A: the N x N sum of the blocks' partials into host memory, made exactly Hermitian;
    // the kernels and the copy run on stream q, and the host waits for them
    auto gram = [&](const char* A, std::vector<cd>& G, cudaStream_t q) -> int {
        // tile buffers; the final reduction reuses them (N x N double2 fit in one buffer)
        launch_pdl(block_gram_kernel, g_gram, t_gram, kGramStages * gtile, q, f4(A), stride4, M, N, partial);
        launch_pdl(gram_final_kernel, (N * N + 7) / 8, 256, 0, q, partial, g_gram, N, Gd);
        if (cudaMemcpyAsync(hostbuf, Gd, sizeof(double2) * N * N, cudaMemcpyDeviceToHost, q) != cudaSuccess ||
            cudaStreamSynchronize(q) != cudaSuccess)
            return LQ_ERR_CUDA;
        G.resize(N * N);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const double2 v = hostbuf[i <= j ? i * N + j : j * N + i];
                G[i * N + j] = i <= j ? cd(v.x, v.y) : cd(v.x, -v.y);
            }
        return LQ_OK;
    };
    // an N x N matrix to the device (through hostbuf: every gram() synchronises the stream before the
    // host writes hostbuf again, so the copy has been made by then)
    auto upload = [&](const std::vector<cd>& Mx) -> int {
        float2* hf = reinterpret_cast<float2*>(hostbuf);
        for (int e = 0; e < N * N; ++e) hf[e] = make_float2((float)Mx[e].real(), (float)Mx[e].imag());
        return cudaMemcpyAsync(Md, hf, mat, cudaMemcpyHostToDevice, s) == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
    };

    // X = 0, R = B, P = R
    if (cudaMemsetAsync(X, 0, stride * N, s) != cudaSuccess ||
        cudaMemcpyAsync(R, Bv, stride * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(P, Bv, stride * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    std::vector<cd> rho, rho0, delta, alpha, beta, rhonew;
    int rc = gram(R, rho, s);
    if (rc) return rc;
    rho0 = rho;
    int it = 0;
    for (; it < maxiter; ++it) {
        bool done = true;
        for (int j = 0; j < N; ++j) done = done && rho[j * N + j].real() <= tol * tol * rho0[j * N + j].real();
        if (done) break;
        // T = K P; then Delta = P^dag A P = T^dag T on s2 while Q = K^dag T runs on s.  The host
        // waits for Delta only (the Gram kernels read T, which the K^dag stage only reads too; s2's
        // copy into hostbuf comes after s's last use of it, which precedes K P in s)
        if ((rc = ops.apply(ops.ctx, Q, P, 0))) return rc;
        if (cudaEventRecord(kdone, s) != cudaSuccess || cudaStreamWaitEvent(s2, kdone, 0) != cudaSuccess)
            return LQ_ERR_CUDA;
        if ((rc = ops.apply(ops.ctx, Q, P, 1))) return rc;
        if ((rc = gram(ops.kimage, delta, s2))) return rc;
        // s2 is idle from here on: s's next Gram may overwrite partial and Gd
        if (!chol_solve(delta, rho, alpha, N)) break;  // block lost rank: hand back to the outer loop
        if ((rc = upload(alpha))) return rc;
        // X += P alpha ; R -= Q alpha
        launch_pdl(block_update_kernel, g_upd, nthr, s_upd, s, w4(X), f4(P), w4(R), f4(Q), stride4, M, N, Md);
        if ((rc = gram(R, rhonew, s))) return rc;
        if (!chol_solve(rho, rhonew, beta, N)) {
            ++it;
            break;
        }
        if ((rc = upload(beta))) return rc;
        // P = R + P beta
        launch_pdl(block_pupdate_kernel, g_pup, nthr, s_pup, s, w4(P), f4(R), stride4, M, N, Md);
        rho = rhonew;
    }
    *iters = it;
    return cudaGetLastError() == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
}

}  // namespace lq
