// convert.cu -- layout and precision conversions: the documented site-major
// exchange layout <-> the native structure-of-arrays blocks the hop streams,
// precision changes between native fields, and gauge-link packing (with the
// optional two-row compression).  The paper's Gridarray layout (Sec. 3.1)
// keeps one degree of freedom of many sites contiguous so that whole SIMD
// registers load at once; the native layout does the same for a warp.
#include <algorithm>
#include <cstring>

#include "lqcd_kernels.h"

namespace lq {

namespace {

template <int SP>
__device__ __forceinline__ void load_sm(const void* base, size_t site, cplx<double> (&s)[12]) {
    if constexpr (SP == LQ_F64) {
        const double2* q = reinterpret_cast<const double2*>(base) + site * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = q[k];
            s[k] = {v.x, v.y};
        }
    } else {
        const float2* q = reinterpret_cast<const float2*>(base) + site * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 v = q[k];
            s[k] = {(double)v.x, (double)v.y};
        }
    }
}

template <int SP>
__device__ __forceinline__ void store_sm(void* base, size_t site, const cplx<double> (&s)[12]) {
    if constexpr (SP == LQ_F64) {
        double2* q = reinterpret_cast<double2*>(base) + site * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = make_double2(s[k].re, s[k].im);
    } else {
        float2* q = reinterpret_cast<float2*>(base) + site * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = make_float2((float)s[k].re, (float)s[k].im);
    }
}

__device__ __forceinline__ size_t lexi_of(const Geom& g, int cb, int p) {
    int x[4];
    cb_coords(g, cb, p, x);
    return (size_t)x[0] + (size_t)g.L[0] * (x[1] + (size_t)g.L[1] * (x[2] + (size_t)g.L[2] * x[3]));
}

// grid.y = rhs * nparity + parity index
template <int DP, int SP, bool TO_NATIVE>
__global__ void spinor_layout_kernel(char* nat, void* sm, Geom g, bool full, int parity, int nparity) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    const int pi = blockIdx.y % nparity;
    const int rhs = blockIdx.y / nparity;
    const int p = full ? pi : parity;
    const size_t nsites_sm = full ? 2 * (size_t)g.Vh : (size_t)g.Vh;
    const size_t site = (size_t)rhs * nsites_sm + (full ? lexi_of(g, i, p) : (size_t)i);
    char* blk = nat + ((size_t)rhs * nparity + pi) * (size_t)spinor_site_bytes(DP) * g.Vh;
    cplx<double> s[12];
    if constexpr (TO_NATIVE) {
        load_sm<SP>(sm, site, s);
        store_spinor<DP, double>(blk, g.Vh, i, s);
    } else {
        load_spinor<DP, double>(blk, g.Vh, i, s);
        store_sm<SP>(sm, site, s);
    }
}

template <int DP, int SP>
__global__ void native_convert_kernel(char* dst, const char* src, int Vh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vh) return;
    const char* sb = src + (size_t)blockIdx.y * spinor_site_bytes(SP) * Vh;
    char* db = dst + (size_t)blockIdx.y * spinor_site_bytes(DP) * Vh;
    cplx<float> sf[12];
    cplx<double> sd[12];
    if constexpr (SP == LQ_F64 || DP == LQ_F64) {
        load_spinor<SP, double>(sb, Vh, i, sd);
        store_spinor<DP, double>(db, Vh, i, sd);
    } else {
        load_spinor<SP, float>(sb, Vh, i, sf);
        store_spinor<DP, float>(db, Vh, i, sf);
    }
}

template <int DP, bool R12, int SP>
__global__ void links_kernel(char* dst, const void* src, Geom g, size_t link_block) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    const int p = blockIdx.y;
    const size_t site = lexi_of(g, i, p);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        cplx<double> u[9];
        const size_t base = (site * 4 + mu) * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if constexpr (SP == LQ_F64) {
                double2 v = reinterpret_cast<const double2*>(src)[base + k];
                u[k] = {v.x, v.y};
            } else {
                float2 v = reinterpret_cast<const float2*>(src)[base + k];
                u[k] = {(double)v.x, (double)v.y};
            }
        }
        store_link<DP, R12>(dst + (size_t)(p * 4 + mu) * link_block, g.Vh, i, u);
    }
}

constexpr int kBlock = 128;

// Largest deviation of a link from SU(3): max over the entries of |U^dag U - 1|
// and |det U - 1|, in FP64.  Two-row compression rebuilds row 3 as
// conj(row 1 x row 2), which is row 3 only for a special unitary matrix.
template <int SP>
__global__ void link_su3_deviation_kernel(const void* src, long nlinks, unsigned long long* out) {
    double dev = 0.0;
    for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (long)gridDim.x * blockDim.x) {
        cplx<double> u[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if constexpr (SP == LQ_F64) {
                const double2 v = reinterpret_cast<const double2*>(src)[l * 9 + k];
                u[k] = {v.x, v.y};
            } else {
                const float2 v = reinterpret_cast<const float2*>(src)[l * 9 + k];
                u[k] = {(double)v.x, (double)v.y};
            }
        }
        // d = the largest |.| seen; fmax would drop a NaN, so NaNs are tracked in nan_seen
        double d = 0.0;
        bool nan_seen = false;
        auto take = [&](cplx<double> z) {
            const double v = sqrt(z.re * z.re + z.im * z.im);
            nan_seen = nan_seen || !(v == v);
            d = v > d ? v : d;
        };
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                cplx<double> g = {i == j ? -1.0 : 0.0, 0.0};  // (U^dag U)_ij - delta_ij
#pragma unroll
                for (int k = 0; k < 3; ++k) cmac_conj(g, u[3 * k + i], u[3 * k + j]);
                take(g);
            }
        }
        // det U by the first row's cofactors
        cplx<double> m0 = {0, 0}, m1 = {0, 0}, m2 = {0, 0};
        cmac(m0, u[4], u[8]);
        cmac(m0, cneg(u[5]), u[7]);
        cmac(m1, u[5], u[6]);
        cmac(m1, cneg(u[3]), u[8]);
        cmac(m2, u[3], u[7]);
        cmac(m2, cneg(u[4]), u[6]);
        cplx<double> det = {-1.0, 0.0};
        cmac(det, u[0], m0);
        cmac(det, u[1], m1);
        cmac(det, u[2], m2);
        take(det);
        if (nan_seen) d = __longlong_as_double(0x7ff0000000000000LL);  // NaN counts as infinitely far
        dev = fmax(dev, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(dev));
}

}  // namespace

#define LQ_DP_SWITCH(dp, BODY)                              \
    switch (dp) {                                           \
    case LQ_F64: { constexpr int DP = LQ_F64; BODY; } break; \
    case LQ_F32: { constexpr int DP = LQ_F32; BODY; } break; \
    case LQ_F16: { constexpr int DP = LQ_F16; BODY; } break; \
    default: { constexpr int DP = LQ_BF16; BODY; } break;    \
    }

cudaError_t launch_spinor_to_native(int dst_prec, void* dst, int src_prec, const void* src, const Geom& g, bool full,
                                    int parity, int nrhs, cudaStream_t st) {
    const int np = full ? 2 : 1;
    dim3 grid((g.Vh + kBlock - 1) / kBlock, nrhs * np);
    char* d = static_cast<char*>(dst);
    void* s = const_cast<void*>(src);
    if (src_prec == LQ_F64) {
        LQ_DP_SWITCH(dst_prec, (spinor_layout_kernel<DP, LQ_F64, true><<<grid, kBlock, 0, st>>>(d, s, g, full, parity, np)))
    } else {
        LQ_DP_SWITCH(dst_prec, (spinor_layout_kernel<DP, LQ_F32, true><<<grid, kBlock, 0, st>>>(d, s, g, full, parity, np)))
    }
    return cudaGetLastError();
}

cudaError_t launch_spinor_from_native(int dst_prec, void* dst, int src_prec, const void* src, const Geom& g,
                                      bool full, int parity, int nrhs, cudaStream_t st) {
    const int np = full ? 2 : 1;
    dim3 grid((g.Vh + kBlock - 1) / kBlock, nrhs * np);
    char* n = const_cast<char*>(static_cast<const char*>(src));
    if (dst_prec == LQ_F64) {
        LQ_DP_SWITCH(src_prec, (spinor_layout_kernel<DP, LQ_F64, false><<<grid, kBlock, 0, st>>>(n, dst, g, full, parity, np)))
    } else {
        LQ_DP_SWITCH(src_prec, (spinor_layout_kernel<DP, LQ_F32, false><<<grid, kBlock, 0, st>>>(n, dst, g, full, parity, np)))
    }
    return cudaGetLastError();
}

cudaError_t launch_native_convert(int dst_prec, void* dst, int src_prec, const void* src, int Vh, int nblocks,
                                  cudaStream_t st) {
    dim3 grid((Vh + kBlock - 1) / kBlock, nblocks);
    char* d = static_cast<char*>(dst);
    const char* s = static_cast<const char*>(src);
#define LQ_SP_CASE(SPV)                                                                         \
    case SPV: {                                                                                 \
        LQ_DP_SWITCH(dst_prec, (native_convert_kernel<DP, SPV><<<grid, kBlock, 0, st>>>(d, s, Vh))) \
    } break;
    switch (src_prec) {
        LQ_SP_CASE(LQ_F64)
        LQ_SP_CASE(LQ_F32)
        LQ_SP_CASE(LQ_F16)
        LQ_SP_CASE(LQ_BF16)
    }
#undef LQ_SP_CASE
    return cudaGetLastError();
}

cudaError_t launch_links_to_native(int dst_prec, bool r12, void* dst, int src_prec, const void* src, const Geom& g,
                                   cudaStream_t st) {
    dim3 grid((g.Vh + kBlock - 1) / kBlock, 2);
    const size_t lb = (size_t)link_site_bytes(dst_prec, r12) * g.Vh;
    char* d = static_cast<char*>(dst);
    if (src_prec == LQ_F64) {
        if (r12) { LQ_DP_SWITCH(dst_prec, (links_kernel<DP, true, LQ_F64><<<grid, kBlock, 0, st>>>(d, src, g, lb))) }
        else { LQ_DP_SWITCH(dst_prec, (links_kernel<DP, false, LQ_F64><<<grid, kBlock, 0, st>>>(d, src, g, lb))) }
    } else {
        if (r12) { LQ_DP_SWITCH(dst_prec, (links_kernel<DP, true, LQ_F32><<<grid, kBlock, 0, st>>>(d, src, g, lb))) }
        else { LQ_DP_SWITCH(dst_prec, (links_kernel<DP, false, LQ_F32><<<grid, kBlock, 0, st>>>(d, src, g, lb))) }
    }
    return cudaGetLastError();
}

cudaError_t link_su3_deviation(int src_prec, const void* src, long nlinks, double* dev, cudaStream_t st) {
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(*d));
    if (e != cudaSuccess) return e;
    unsigned long long v = 0;
    e = cudaMemsetAsync(d, 0, sizeof(*d), st);
    const int grid = (int)std::min<long>((nlinks + 255) / 256, 4096);
    if (e == cudaSuccess && nlinks > 0) {
        if (src_prec == LQ_F64) link_su3_deviation_kernel<LQ_F64><<<grid, 256, 0, st>>>(src, nlinks, d);
        else link_su3_deviation_kernel<LQ_F32><<<grid, 256, 0, st>>>(src, nlinks, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    std::memcpy(dev, &v, sizeof(v));
    return e;
}

}  // namespace lq
