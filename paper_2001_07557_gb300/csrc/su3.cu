// su3.cu -- the lattice-wide colour-matrix product C[x] = A[x] B[x] of the
// paper's SU(3) matrix-matrix benchmark (Sec. 3.3, Fig. 4a-c).
//
// Layout: n 3x3 complex matrices [x][row][col]{re, im}, the paper's array of
// two-element structures; 144 bytes per FP64 matrix, 72 per FP32 matrix.
// A persistent block walks tiles of TS consecutive matrices:
//   * one thread moves the tile of A and the tile of B into one of two
//     shared-memory stages with bulk asynchronous copies (cp.async.bulk, the
//     one-dimensional TMA path), which complete on that stage's mbarrier;
//     the copies of the next tile are in flight while this one is multiplied;
//   * thread t multiplies matrix t of the tile.  Its shared-memory reads have
//     a stride of 72 or 144 bytes, which touches every bank once per phase;
//   * the products go to one of two output buffers, which one thread writes
//     back with a bulk store.
// FP32 is bound by HBM bandwidth (216 bytes and 198 flop per matrix).  FP64
// is bound by the FP64 units: 198 flop take longer at GB300's FP64 rate than
// its 432 bytes take to move.  Every barrier wait is bounded; a wait that runs
// out is counted in g_wait_timeouts and its block stops.  Before it returns,
// the block waits (bounded again) for the copies it issued into its other
// stage, and for its bulk stores, so that no copy into its shared memory is
// left in flight.  The copies of the stage whose wait ran out are not waited
// for a second time: that wait already lasted about a second, while a tile's
// copies take microseconds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "lqcd.h"
#include "trace.h"

namespace lq {

__device__ unsigned g_wait_timeouts;

namespace {

template <typename T>
struct Cx2;
template <>
struct Cx2<double> {
    using type = double2;
};
template <>
struct Cx2<float> {
    using type = float2;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Poll the barrier's phase; false once about a second has passed without
// completion (the iteration cap is a second bound should the timer stall).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    for (int i = 0; i < (1 << 26); ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 255) == 255 && globaltimer_ns() - t0 > 1000000000ull) return false;
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}

template <typename T2>
__device__ __forceinline__ void su3_product(const T2 (&a)[9], const T2 (&b)[9], T2 (&c)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T2 s;
            s.x = a[3 * i].x * b[j].x - a[3 * i].y * b[j].y;
            s.y = a[3 * i].x * b[j].y + a[3 * i].y * b[j].x;
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                s.x = fma(a[3 * i + k].x, b[3 * k + j].x, s.x);
                s.x = fma(-a[3 * i + k].y, b[3 * k + j].y, s.x);
                s.y = fma(a[3 * i + k].x, b[3 * k + j].y, s.y);
                s.y = fma(a[3 * i + k].y, b[3 * k + j].x, s.y);
            }
            c[3 * i + j] = s;
        }
    }
}

// Shared memory: stage s holds the tile of A at 2*s*TB and of B at (2*s+1)*TB,
// output buffer o at (4+o)*TB, the two stage barriers at 6*TB.
template <typename T, int TS>
struct Su3Cfg {
    using T2 = typename Cx2<T>::type;
    static constexpr int MB = 9 * (int)sizeof(T2);  // bytes per matrix
    static constexpr int TB = TS * MB;              // bytes per tile
    static constexpr int SMEM = 6 * TB + 16;
};

// stall != 0 (testing only) arms each stage barrier for 16 more bytes than its
// copies bring, so that the bounded wait runs out.
template <typename T, int TS>
__global__ void __launch_bounds__(TS) su3_mul_kernel(const char* A, const char* B, char* C, long n, int stall) {
    using Cfg = Su3Cfg<T, TS>;
    using T2 = typename Cfg::T2;
    constexpr int MB = Cfg::MB, TB = Cfg::TB;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ int s_ok;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 6 * TB);
    const int t = threadIdx.x;
    const long ntiles = (n + TS - 1) / TS;
    // matrices of a tile, and those moved by the bulk copies: a bulk copy moves a
    // multiple of 16 bytes, so an odd last FP32 matrix goes by plain loads and stores
    auto count = [&](long tile) { return (int)(n - tile * TS < TS ? n - tile * TS : TS); };
    auto bulk = [&](int cnt) { return (sizeof(T) == 4 && (cnt & 1)) ? cnt - 1 : cnt; };
    auto issue = [&](long tile, int s) {
        const uint32_t bytes = (uint32_t)bulk(count(tile)) * MB;
        const uint32_t bar = smem_u32(&bars[s]);
        mbar_arrive_expect_tx(bar, 2 * bytes + (stall ? 16u : 0u));
        if (bytes) {
            bulk_load(smem_u32(sm + 2 * s * TB), A + tile * TB, bytes, bar);
            bulk_load(smem_u32(sm + (2 * s + 1) * TB), B + tile * TB, bytes, bar);
        }
    };
    if (t == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < 2; ++s) {
            const long tile = blockIdx.x + (long)s * gridDim.x;
            if (tile < ntiles) issue(tile, s);
        }
    }
    int it = 0;
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it & 1;
        if (t == 0) {
            const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((it >> 1) & 1));
            if (!ok) atomicAdd(&g_wait_timeouts, 1u);
            s_ok = ok;
        }
        __syncthreads();  // the tile is visible to every thread (or the wait ran out)
        if (!s_ok) {
            // drain the other stage: its tile's copies were issued one iteration ago
            if (t == 0 && tile + gridDim.x < ntiles &&
                !mbar_wait_bounded(smem_u32(&bars[s ^ 1]), (uint32_t)(((it + 1) >> 1) & 1)))
                atomicAdd(&g_wait_timeouts, 1u);
            break;
        }
        const int cnt = count(tile), nb = bulk(cnt);
        unsigned char* cbuf = sm + (4 + (it & 1)) * TB;
        if (t < cnt) {
            T2 a[9], b[9], c[9];
            const T2* pa = t < nb ? reinterpret_cast<const T2*>(sm + 2 * s * TB + t * MB)
                                  : reinterpret_cast<const T2*>(A + (tile * TS + t) * MB);
            const T2* pb = t < nb ? reinterpret_cast<const T2*>(sm + (2 * s + 1) * TB + t * MB)
                                  : reinterpret_cast<const T2*>(B + (tile * TS + t) * MB);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                a[k] = pa[k];
                b[k] = pb[k];
            }
            su3_product(a, b, c);
            T2* pc = t < nb ? reinterpret_cast<T2*>(cbuf + t * MB) : reinterpret_cast<T2*>(C + (tile * TS + t) * MB);
#pragma unroll
            for (int k = 0; k < 9; ++k) pc[k] = c[k];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // C buffer -> bulk-store reads
        __syncthreads();  // every thread is done with stage s and has written the C buffer
        if (t == 0) {
            if (nb) bulk_store(C + tile * TB, smem_u32(cbuf), (uint32_t)nb * MB);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            const long next = tile + 2L * gridDim.x;
            if (next < ntiles) issue(next, s);
            // the store issued one iteration ago has read the buffer the next iteration fills
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        }
    }
    if (t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <typename T, int TS>
int launch_su3(void* C, const void* A, const void* B, long n, cudaStream_t st, int stall = 0) {
    using Cfg = Su3Cfg<T, TS>;
    auto kern = su3_mul_kernel<T, TS>;
    static int grid_max = 0;  // resident blocks on this device, found once
    if (!grid_max) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TS, Cfg::SMEM) != cudaSuccess)
            return LQ_ERR_CUDA;
        grid_max = std::max(1, sms * std::max(per_sm, 1));
    }
    const long ntiles = (n + TS - 1) / TS;
    const int grid = (int)std::min<long>(ntiles, grid_max);
    kern<<<grid, TS, Cfg::SMEM, st>>>(static_cast<const char*>(A), static_cast<const char*>(B),
                                      static_cast<char*>(C), n, stall);
    return cudaGetLastError() == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
}

bool overlaps(const void* p, const void* q, size_t bytes) {
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + bytes && b < a + bytes;
}

}  // namespace
}  // namespace lq

extern "C" {

int lq_su3_mul(void* C, const void* A, const void* B, long n, int fmt, void* stream) {
    lq::TraceRange trace_("lqcd/su3_mul");
    if (n < 0 || (fmt != LQ_F64 && fmt != LQ_F32)) return LQ_ERR_ARG;
    if (n == 0) return LQ_OK;
    if (!A || !B || !C) return LQ_ERR_ARG;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15) return LQ_ERR_LAYOUT;
    const size_t bytes = (size_t)n * (fmt == LQ_F64 ? 144 : 72);
    if ((C != A && lq::overlaps(C, A, bytes)) || (C != B && lq::overlaps(C, B, bytes))) return LQ_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return fmt == LQ_F64 ? lq::launch_su3<double, 128>(C, A, B, n, st) : lq::launch_su3<float, 256>(C, A, B, n, st);
}

int lq_test_stalled_wait(void) {
    // one tile of zero matrices, product kernel with its barrier armed for bytes that never come
    const long n = 256;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 3 * 72 * n) != cudaSuccess) {
        cudaGetLastError();
        return LQ_ERR_NOMEM;
    }
    char* p = static_cast<char*>(buf);
    int rc = cudaMemset(buf, 0, 3 * 72 * n) == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
    if (rc == LQ_OK) rc = lq::launch_su3<float, 256>(p + 2 * 72 * n, p, p + 72 * n, n, nullptr, 1);
    if (rc == LQ_OK && cudaDeviceSynchronize() != cudaSuccess) rc = LQ_ERR_CUDA;
    cudaFree(buf);
    return rc;
}

int lq_wait_timeouts(unsigned* count) {
    if (!count) return LQ_ERR_ARG;
    unsigned v = 0;
    const unsigned zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&v, lq::g_wait_timeouts, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(lq::g_wait_timeouts, &zero, sizeof zero) != cudaSuccess)
        return LQ_ERR_CUDA;
    *count = v;
    return v ? LQ_ERR_TIMEOUT : LQ_OK;
}

}  // extern "C"
