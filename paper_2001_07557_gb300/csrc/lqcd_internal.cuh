// lqcd_internal.cuh -- device-side building blocks of the Wilson hop:
// lattice geometry, native-layout loads/stores in every storage precision,
// chiral-basis spin projection / reconstruction, SU(3) x half-spinor products.
//
// Operator conventions (the paper names the Wilson Dirac operator, Sec. 3.3,
// Fig. 4d, without writing it): H psi(x) = sum_mu (1 - gamma_mu) U_mu(x)
// psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu), chiral basis
// gamma_mu = [[0, A_mu], [A_mu^dag, 0]] with A_k = -i sigma_k, A_t = 1.
// Then (1 + s gamma_mu) psi = [h; s A_mu^dag h] with h = psi_up + s A_mu psi_dn,
// so each hop needs one 2-spin x 3-colour half spinor (the rank-2 projector
// of r = 1), two 3x3 complex products, and a reconstruction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "lqcd.h"

namespace lq {

// ------------------------------------------------------------------ geometry

struct Geom {
    int L[4];   // L0..L3
    int Lh0;    // L0 / 2
    int Vh;     // sites per parity
    int bc[4];  // +1 / -1 boundary phase per direction
    // exact division by Lh0, L1, L2: q = (n * m) >> 40 with m = floor(2^40 / d) + 1,
    // exact for n * d < 2^40 (here n < 2^27 and d <= 2^13)
    unsigned long long mLh0, mL1, mL2;
};

__host__ __device__ inline unsigned long long div_magic(int d) { return ((1ULL << 40) / (unsigned)d) + 1ULL; }

__device__ __forceinline__ int fast_div(int n, unsigned long long m) {
    return (int)(((unsigned long long)(unsigned)n * m) >> 40);
}

// Coordinates of the site with checkerboard index cb and parity p.
__device__ __forceinline__ void cb_coords(const Geom& g, int cb, int p, int x[4]) {
    const int t1 = fast_div(cb, g.mLh0);
    const int xh = cb - t1 * g.Lh0;
    const int t2 = fast_div(t1, g.mL1);
    x[1] = t1 - t2 * g.L[1];
    x[3] = fast_div(t2, g.mL2);
    x[2] = t2 - x[3] * g.L[2];
    x[0] = 2 * xh + ((p + x[1] + x[2] + x[3]) & 1);
}

// Device-resident CG scalars of one right-hand side.
struct CgScalars {
    double rr;     // |r|^2
    double bb;     // |b|^2
    double stop2;  // tol^2 |b|^2
    double pAp;
    double alpha;
    double beta;
    int iter;
    int maxiter;
    int done;      // converged, broke down, or out of iterations
    int status;    // LQ_OK / LQ_ERR_BREAKDOWN / LQ_ERR_NOT_CONVERGED / LQ_ERR_NAN
};

// ------------------------------------------------------ index-checked build
// Built with -DLQ_INDEX_CHECK (build.build(checked=True)), the hop kernels
// compare every neighbour and site index they compute with the parity block
// before using it.  An index out of range is counted in the translation unit's
// counter (the first one kept) and replaced by 0, so that the check itself
// cannot fault; lq_index_faults reads and clears the counters.  The normal
// build compiles the check away.  (It stands in for a memory checker, which
// this build does not run on the GPU.)
#ifdef LQ_INDEX_CHECK
static __device__ unsigned long long lq_index_fault_count;
static __device__ long long lq_index_fault_first;
__device__ __forceinline__ int check_site(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    if (atomicAdd(&lq_index_fault_count, 1ull) == 0ull) lq_index_fault_first = i;
    return 0;
}
// host reader of this translation unit's counter: returns the count (~0 on a CUDA
// error), sets *first to the first bad index when the count is not zero, clears it
#define LQ_INDEX_FAULTS_READER(name)                                                          \
    unsigned long long name(long long* first) {                                               \
        unsigned long long c = 0;                                                             \
        long long f = -1;                                                                     \
        const unsigned long long z = 0;                                                       \
        if (cudaMemcpyFromSymbol(&c, lq_index_fault_count, sizeof(c)) != cudaSuccess ||       \
            cudaMemcpyFromSymbol(&f, lq_index_fault_first, sizeof(f)) != cudaSuccess ||       \
            cudaMemcpyToSymbol(lq_index_fault_count, &z, sizeof(z)) != cudaSuccess)           \
            return ~0ull;                                                                     \
        if (first && c) *first = f;                                                           \
        return c;                                                                             \
    }
#else
__device__ __forceinline__ int check_site(int i, int) { return i; }
#define LQ_INDEX_FAULTS_READER(name) \
    unsigned long long name(long long*) { return 0; }
#endif

// ------------------------------------------------------------------ complex

template <typename T>
struct cplx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cmul_i(cplx<T> a) { return {-a.im, a.re}; }  // i a
template <typename T>
__device__ __forceinline__ cplx<T> cneg(cplx<T> a) { return {-a.re, -a.im}; }

// a + S*b for a compile-time sign S
template <int S, typename T>
__device__ __forceinline__ cplx<T> cadds(cplx<T> a, cplx<T> b) {
    if constexpr (S > 0) return cadd(a, b);
    else return csub(a, b);
}

// acc += a * b
template <typename T>
__device__ __forceinline__ void cmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename T>
__device__ __forceinline__ void cmac_conj(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// ----------------------------------------------------- storage precisions

template <int P>
struct Prec;
template <>
struct Prec<LQ_F64> {
    using real = double;
    static constexpr int spinor_bytes = 192;  // 12 planes x 16 B
    static constexpr bool has_norm = false;
};
template <>
struct Prec<LQ_F32> {
    using real = float;
    static constexpr int spinor_bytes = 96;  // 6 planes x 16 B
    static constexpr bool has_norm = false;
};
template <>
struct Prec<LQ_F16> {
    using real = float;
    static constexpr int spinor_bytes = 52;  // 3 planes x 16 B + 4 B norm
    static constexpr bool has_norm = true;
};
template <>
struct Prec<LQ_BF16> {
    using real = float;
    static constexpr int spinor_bytes = 52;
    static constexpr bool has_norm = true;
};

// Link planes per (parity, mu) block: bytes of one site's link.
__host__ __device__ constexpr int link_site_bytes(int prec, bool r12) {
    return prec == LQ_F64 ? (r12 ? 96 : 144) : prec == LQ_F32 ? (r12 ? 48 : 72) : (r12 ? 24 : 36);
}
__host__ __device__ constexpr int spinor_site_bytes(int prec) {
    return prec == LQ_F64 ? 192 : prec == LQ_F32 ? 96 : 52;
}

// two 16-bit values <-> float2
__device__ __forceinline__ float2 h2f(uint32_t v, std::integral_constant<int, LQ_F16>) {
    __half2 h = *reinterpret_cast<__half2*>(&v);
    return __half22float2(h);
}
__device__ __forceinline__ float2 h2f(uint32_t v, std::integral_constant<int, LQ_BF16>) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
    return __bfloat1622float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b, std::integral_constant<int, LQ_F16>) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b, std::integral_constant<int, LQ_BF16>) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------ spinor access
// A parity block of Vh sites; s[k] = complex number k = (spin k/3, colour k%3).

template <int P, typename T>
__device__ __forceinline__ void load_spinor(const char* __restrict__ blk, int Vh, int i, cplx<T> (&s)[12]) {
    if constexpr (P == LQ_F64) {
        const double2* q = reinterpret_cast<const double2*>(blk);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = __ldg(q + (size_t)k * Vh + i);
            s[k] = {(T)v.x, (T)v.y};
        }
    } else if constexpr (P == LQ_F32) {
        const float4* q = reinterpret_cast<const float4*>(blk);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = __ldg(q + (size_t)k * Vh + i);
            s[2 * k] = {(T)v.x, (T)v.y};
            s[2 * k + 1] = {(T)v.z, (T)v.w};
        }
    } else {
        const uint4* q = reinterpret_cast<const uint4*>(blk);
        const float nrm = __ldg(reinterpret_cast<const float*>(blk + (size_t)48 * Vh) + i);
        std::integral_constant<int, P> tag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(q + (size_t)k * Vh + i);
            float2 a = h2f(v.x, tag), b = h2f(v.y, tag), c = h2f(v.z, tag), d = h2f(v.w, tag);
            s[4 * k + 0] = {a.x * nrm, a.y * nrm};
            s[4 * k + 1] = {b.x * nrm, b.y * nrm};
            s[4 * k + 2] = {c.x * nrm, c.y * nrm};
            s[4 * k + 3] = {d.x * nrm, d.y * nrm};
        }
    }
}

// As load_spinor, but FP16/BF16 values are returned unscaled with the site
// norm in `nrm` (1 for FP32/FP64), so that the norm can ride on later FMAs.
template <int P, typename T>
__device__ __forceinline__ void load_spinor_raw(const char* __restrict__ blk, int Vh, int i, cplx<T> (&s)[12],
                                                T& nrm) {
    if constexpr (P == LQ_F64 || P == LQ_F32) {
        load_spinor<P, T>(blk, Vh, i, s);
        nrm = (T)1;
    } else {
        const uint4* q = reinterpret_cast<const uint4*>(blk);
        nrm = __ldg(reinterpret_cast<const float*>(blk + (size_t)48 * Vh) + i);
        std::integral_constant<int, P> tag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(q + (size_t)k * Vh + i);
            float2 a = h2f(v.x, tag), b = h2f(v.y, tag), c = h2f(v.z, tag), d = h2f(v.w, tag);
            s[4 * k + 0] = {a.x, a.y};
            s[4 * k + 1] = {b.x, b.y};
            s[4 * k + 2] = {c.x, c.y};
            s[4 * k + 3] = {d.x, d.y};
        }
    }
}

template <int P, typename T>
__device__ __forceinline__ void store_spinor(char* __restrict__ blk, int Vh, int i, const cplx<T> (&s)[12]) {
    if constexpr (P == LQ_F64) {
        double2* q = reinterpret_cast<double2*>(blk);
#pragma unroll
        for (int k = 0; k < 12; ++k) q[(size_t)k * Vh + i] = make_double2((double)s[k].re, (double)s[k].im);
    } else if constexpr (P == LQ_F32) {
        float4* q = reinterpret_cast<float4*>(blk);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            q[(size_t)k * Vh + i] =
                make_float4((float)s[2 * k].re, (float)s[2 * k].im, (float)s[2 * k + 1].re, (float)s[2 * k + 1].im);
    } else {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf((float)s[k].re), fabsf((float)s[k].im)));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4* q = reinterpret_cast<uint4*>(blk);
        std::integral_constant<int, P> tag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v;
            v.x = f2h((float)s[4 * k + 0].re * inv, (float)s[4 * k + 0].im * inv, tag);
            v.y = f2h((float)s[4 * k + 1].re * inv, (float)s[4 * k + 1].im * inv, tag);
            v.z = f2h((float)s[4 * k + 2].re * inv, (float)s[4 * k + 2].im * inv, tag);
            v.w = f2h((float)s[4 * k + 3].re * inv, (float)s[4 * k + 3].im * inv, tag);
            q[(size_t)k * Vh + i] = v;
        }
        reinterpret_cast<float*>(blk + (size_t)48 * Vh)[i] = m;
    }
}

// -------------------------------------------------------------- link access
// One (parity, mu) block of Vh links.  u[3*row + col].

template <typename T>
__device__ __forceinline__ void reconstruct_row2(cplx<T> (&u)[9]) {
    // row2 = conj(row0 x row1) for a special unitary matrix
    u[6] = {u[1].re * u[5].re - u[1].im * u[5].im - (u[2].re * u[4].re - u[2].im * u[4].im),
            -(u[1].re * u[5].im + u[1].im * u[5].re - (u[2].re * u[4].im + u[2].im * u[4].re))};
    u[7] = {u[2].re * u[3].re - u[2].im * u[3].im - (u[0].re * u[5].re - u[0].im * u[5].im),
            -(u[2].re * u[3].im + u[2].im * u[3].re - (u[0].re * u[5].im + u[0].im * u[5].re))};
    u[8] = {u[0].re * u[4].re - u[0].im * u[4].im - (u[1].re * u[3].re - u[1].im * u[3].im),
            -(u[0].re * u[4].im + u[0].im * u[4].re - (u[1].re * u[3].im + u[1].im * u[3].re))};
}

// Link record of one site: NC complex numbers (9, or the first two rows = 6
// with compression) of ESZ bytes each, stored as NFULL 16-byte planes and,
// when the record is not a multiple of 16 bytes, one TAIL-byte plane:
//   FP64 18: 9 x 16 B     FP64 12: 6 x 16 B
//   FP32 18: 4 x 16 B + 8 B      FP32 12: 3 x 16 B
//   FP16 18: 2 x 16 B + 4 B      FP16 12: 1 x 16 B + 8 B
// Plane c of a (parity, mu) block starts at c * 16 * Vh, the tail plane at
// NFULL * 16 * Vh; a site's bytes sit at index i within each plane.
template <int P, bool R12>
struct LinkLayout {
    static constexpr int ESZ = P == LQ_F64 ? 16 : P == LQ_F32 ? 8 : 4;
    static constexpr int NC = R12 ? 6 : 9;
    static constexpr int BYTES = NC * ESZ;
    static constexpr int NFULL = BYTES / 16;
    static constexpr int TAIL = BYTES % 16;  // 0, 4 or 8
    static constexpr int WORDS = BYTES / 4;
};

template <int P, bool R12>
struct RawLink {
    uint32_t w[LinkLayout<P, R12>::WORDS];
};

template <int P, bool R12>
__device__ __forceinline__ void raw_load(RawLink<P, R12>& r, const char* __restrict__ blk, int Vh, int i) {
    using LL = LinkLayout<P, R12>;
#pragma unroll
    for (int c = 0; c < LL::NFULL; ++c) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(blk) + (size_t)c * Vh + i);
        r.w[4 * c] = v.x;
        r.w[4 * c + 1] = v.y;
        r.w[4 * c + 2] = v.z;
        r.w[4 * c + 3] = v.w;
    }
    const char* tail = blk + (size_t)LL::NFULL * 16 * Vh;
    if constexpr (LL::TAIL == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(tail) + i);
        r.w[4 * LL::NFULL] = v.x;
        r.w[4 * LL::NFULL + 1] = v.y;
    } else if constexpr (LL::TAIL == 4) {
        r.w[4 * LL::NFULL] = __ldg(reinterpret_cast<const uint32_t*>(tail) + i);
    }
}

template <int P, bool R12, typename T>
__device__ __forceinline__ void raw_unpack(const RawLink<P, R12>& r, cplx<T> (&u)[9]) {
    using LL = LinkLayout<P, R12>;
#pragma unroll
    for (int k = 0; k < LL::NC; ++k) {
        if constexpr (P == LQ_F64) {
            u[k] = {(T)__hiloint2double((int)r.w[4 * k + 1], (int)r.w[4 * k]),
                    (T)__hiloint2double((int)r.w[4 * k + 3], (int)r.w[4 * k + 2])};
        } else if constexpr (P == LQ_F32) {
            u[k] = {(T)__uint_as_float(r.w[2 * k]), (T)__uint_as_float(r.w[2 * k + 1])};
        } else {
            const float2 v = h2f(r.w[k], std::integral_constant<int, P>());
            u[k] = {(T)v.x, (T)v.y};
        }
    }
    if constexpr (R12) reconstruct_row2(u);
}

template <int P, bool R12, typename T>
__device__ __forceinline__ void load_link(const char* __restrict__ blk, int Vh, int i, cplx<T> (&u)[9]) {
    RawLink<P, R12> r;
    raw_load(r, blk, Vh, i);
    raw_unpack<P, R12, T>(r, u);
}

template <int P, bool R12>
__device__ __forceinline__ void store_link(char* __restrict__ blk, int Vh, int i, const cplx<double> (&u)[9]) {
    using LL = LinkLayout<P, R12>;
    RawLink<P, R12> r;
#pragma unroll
    for (int k = 0; k < LL::NC; ++k) {
        if constexpr (P == LQ_F64) {
            r.w[4 * k] = (uint32_t)__double2loint(u[k].re);
            r.w[4 * k + 1] = (uint32_t)__double2hiint(u[k].re);
            r.w[4 * k + 2] = (uint32_t)__double2loint(u[k].im);
            r.w[4 * k + 3] = (uint32_t)__double2hiint(u[k].im);
        } else if constexpr (P == LQ_F32) {
            r.w[2 * k] = __float_as_uint((float)u[k].re);
            r.w[2 * k + 1] = __float_as_uint((float)u[k].im);
        } else {
            r.w[k] = f2h((float)u[k].re, (float)u[k].im, std::integral_constant<int, P>());
        }
    }
#pragma unroll
    for (int c = 0; c < LL::NFULL; ++c)
        reinterpret_cast<uint4*>(blk)[(size_t)c * Vh + i] =
            make_uint4(r.w[4 * c], r.w[4 * c + 1], r.w[4 * c + 2], r.w[4 * c + 3]);
    char* tail = blk + (size_t)LL::NFULL * 16 * Vh;
    if constexpr (LL::TAIL == 8) {
        reinterpret_cast<uint2*>(tail)[i] = make_uint2(r.w[4 * LL::NFULL], r.w[4 * LL::NFULL + 1]);
    } else if constexpr (LL::TAIL == 4) {
        reinterpret_cast<uint32_t*>(tail)[i] = r.w[4 * LL::NFULL];
    }
}

// ----------------------------------------------- raw (packed) neighbour data
// The hop issues the loads of the next direction before it computes the
// current one; holding the data in its packed storage form keeps that
// prefetch cheap in registers (19 words per direction for FP16, 12-real).

template <int P>
struct RawSpinor;
template <>
struct RawSpinor<LQ_F64> {
    double2 v[12];
};
template <>
struct RawSpinor<LQ_F32> {
    float4 v[6];
};
template <>
struct RawSpinor<LQ_F16> {
    uint4 v[3];
    float n;
};
template <>
struct RawSpinor<LQ_BF16> {
    uint4 v[3];
    float n;
};

template <int P>
__device__ __forceinline__ void raw_load(RawSpinor<P>& r, const char* __restrict__ blk, int Vh, int i) {
    if constexpr (P == LQ_F64) {
        const double2* q = reinterpret_cast<const double2*>(blk);
#pragma unroll
        for (int k = 0; k < 12; ++k) r.v[k] = __ldg(q + (size_t)k * Vh + i);
    } else if constexpr (P == LQ_F32) {
        const float4* q = reinterpret_cast<const float4*>(blk);
#pragma unroll
        for (int k = 0; k < 6; ++k) r.v[k] = __ldg(q + (size_t)k * Vh + i);
    } else {
        const uint4* q = reinterpret_cast<const uint4*>(blk);
#pragma unroll
        for (int k = 0; k < 3; ++k) r.v[k] = __ldg(q + (size_t)k * Vh + i);
        r.n = __ldg(reinterpret_cast<const float*>(blk + (size_t)48 * Vh) + i);
    }
}

// values (unscaled for FP16/BF16) and the site norm (1 for FP32/FP64)
template <int P, typename T>
__device__ __forceinline__ void raw_unpack(const RawSpinor<P>& r, cplx<T> (&s)[12], T& nrm) {
    if constexpr (P == LQ_F64) {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = {(T)r.v[k].x, (T)r.v[k].y};
        nrm = (T)1;
    } else if constexpr (P == LQ_F32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            s[2 * k] = {(T)r.v[k].x, (T)r.v[k].y};
            s[2 * k + 1] = {(T)r.v[k].z, (T)r.v[k].w};
        }
        nrm = (T)1;
    } else {
        std::integral_constant<int, P> tag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float2 a = h2f(r.v[k].x, tag), b = h2f(r.v[k].y, tag), c = h2f(r.v[k].z, tag), d = h2f(r.v[k].w, tag);
            s[4 * k + 0] = {a.x, a.y};
            s[4 * k + 1] = {b.x, b.y};
            s[4 * k + 2] = {c.x, c.y};
            s[4 * k + 3] = {d.x, d.y};
        }
        nrm = r.n;
    }
}

// ----------------------------------------------------- spin projection
// (1 + S gamma_mu) psi = [h; S A_mu^dag h], h = psi_up + S A_mu psi_dn.
// h[c] = spin 0 colour c, h[3 + c] = spin 1 colour c.

template <int MU, int S, typename T>
__device__ __forceinline__ void project(const cplx<T> (&s)[12], cplx<T> (&h)[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<T> p0 = s[c], p1 = s[3 + c], p2 = s[6 + c], p3 = s[9 + c];
        if constexpr (MU == 0) {  // A = -i sigma_x: A psi_dn = (-i p3, -i p2)
            h[c] = cadds<-S>(p0, cmul_i(p3));
            h[3 + c] = cadds<-S>(p1, cmul_i(p2));
        } else if constexpr (MU == 1) {  // A = -i sigma_y = [[0,-1],[1,0]]: (-p3, p2)
            h[c] = cadds<-S>(p0, p3);
            h[3 + c] = cadds<S>(p1, p2);
        } else if constexpr (MU == 2) {  // A = -i sigma_z = diag(-i, i): (-i p2, i p3)
            h[c] = cadds<-S>(p0, cmul_i(p2));
            h[3 + c] = cadds<S>(p1, cmul_i(p3));
        } else {  // A = 1
            h[c] = cadds<S>(p0, p2);
            h[3 + c] = cadds<S>(p1, p3);
        }
    }
}

// acc += [uh; S A_mu^dag uh]
template <int MU, int S, typename T>
__device__ __forceinline__ void reconstruct_add(cplx<T> (&acc)[12], const cplx<T> (&uh)[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<T> a = uh[c], b = uh[3 + c];
        acc[c] = cadd(acc[c], a);
        acc[3 + c] = cadd(acc[3 + c], b);
        if constexpr (MU == 0) {  // A^dag = [[0, i],[i, 0]]: (i b, i a)
            acc[6 + c] = cadds<S>(acc[6 + c], cmul_i(b));
            acc[9 + c] = cadds<S>(acc[9 + c], cmul_i(a));
        } else if constexpr (MU == 1) {  // A^dag = [[0, 1],[-1, 0]]: (b, -a)
            acc[6 + c] = cadds<S>(acc[6 + c], b);
            acc[9 + c] = cadds<-S>(acc[9 + c], a);
        } else if constexpr (MU == 2) {  // A^dag = diag(i, -i): (i a, -i b)
            acc[6 + c] = cadds<S>(acc[6 + c], cmul_i(a));
            acc[9 + c] = cadds<-S>(acc[9 + c], cmul_i(b));
        } else {
            acc[6 + c] = cadds<S>(acc[6 + c], a);
            acc[9 + c] = cadds<S>(acc[9 + c], b);
        }
    }
}

// acc += n [uh; S A_mu^dag uh] with a run-time scale n (site norm x boundary phase):
// every term is one FMA, so the scale costs nothing over reconstruct_add.
template <typename T>
__device__ __forceinline__ void cfma(cplx<T>& acc, T n, cplx<T> b) {
    acc.re = fma(n, b.re, acc.re);
    acc.im = fma(n, b.im, acc.im);
}
template <typename T>
__device__ __forceinline__ void cfma_i(cplx<T>& acc, T n, cplx<T> b) {  // acc += n * i b
    acc.re = fma(-n, b.im, acc.re);
    acc.im = fma(n, b.re, acc.im);
}
template <int MU, int S, typename T>
__device__ __forceinline__ void reconstruct_fma(cplx<T> (&acc)[12], const cplx<T> (&uh)[6], T n) {
    const T sn = S > 0 ? n : -n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<T> a = uh[c], b = uh[3 + c];
        cfma(acc[c], n, a);
        cfma(acc[3 + c], n, b);
        if constexpr (MU == 0) {
            cfma_i(acc[6 + c], sn, b);
            cfma_i(acc[9 + c], sn, a);
        } else if constexpr (MU == 1) {
            cfma(acc[6 + c], sn, b);
            cfma(acc[9 + c], -sn, a);
        } else if constexpr (MU == 2) {
            cfma_i(acc[6 + c], sn, a);
            cfma_i(acc[9 + c], -sn, b);
        } else {
            cfma(acc[6 + c], sn, a);
            cfma(acc[9 + c], sn, b);
        }
    }
}

// ------------------------------------------ FP16 / BF16 packed arithmetic
// A complex number held as one 32-bit word: (re, im) = (low, high) 16-bit half.
// The spin projection of an FP16/BF16 spinor is done on packed halves (one
// add per component, rounded to 11 / 8 significant bits like the stored
// inputs), and the SU(3) products multiply the packed halves with the
// mixed-precision FMA (16-bit inputs, FP32 accumulator): no conversion
// instructions, all sums in FP32.

template <int P>
__device__ __forceinline__ uint32_t h2_add(uint32_t a, uint32_t b) {
    if constexpr (P == LQ_F16) {
        __half2 r = __hadd2(*reinterpret_cast<__half2*>(&a), *reinterpret_cast<__half2*>(&b));
        return *reinterpret_cast<uint32_t*>(&r);
    } else {
        __nv_bfloat162 r = __hadd2(*reinterpret_cast<__nv_bfloat162*>(&a), *reinterpret_cast<__nv_bfloat162*>(&b));
        return *reinterpret_cast<uint32_t*>(&r);
    }
}
template <int P>
__device__ __forceinline__ uint32_t h2_sub(uint32_t a, uint32_t b) {
    if constexpr (P == LQ_F16) {
        __half2 r = __hsub2(*reinterpret_cast<__half2*>(&a), *reinterpret_cast<__half2*>(&b));
        return *reinterpret_cast<uint32_t*>(&r);
    } else {
        __nv_bfloat162 r = __hsub2(*reinterpret_cast<__nv_bfloat162*>(&a), *reinterpret_cast<__nv_bfloat162*>(&b));
        return *reinterpret_cast<uint32_t*>(&r);
    }
}
// i z = (-im, re): swap the halves, flip the sign bit of the new low half
__device__ __forceinline__ uint32_t h2_mul_i(uint32_t z) { return __byte_perm(z, 0, 0x1032) ^ 0x00008000u; }
template <int P, int S>
__device__ __forceinline__ uint32_t h2_adds(uint32_t a, uint32_t b) {
    if constexpr (S > 0) return h2_add<P>(a, b);
    else return h2_sub<P>(a, b);
}

// (1 + S gamma_mu) psi projected on packed halves; same algebra as project()
template <int P, int MU, int S>
__device__ __forceinline__ void project_h2(const uint32_t (&s)[12], uint32_t (&h)[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const uint32_t p0 = s[c], p1 = s[3 + c], p2 = s[6 + c], p3 = s[9 + c];
        if constexpr (MU == 0) {
            h[c] = h2_adds<P, -S>(p0, h2_mul_i(p3));
            h[3 + c] = h2_adds<P, -S>(p1, h2_mul_i(p2));
        } else if constexpr (MU == 1) {
            h[c] = h2_adds<P, -S>(p0, p3);
            h[3 + c] = h2_adds<P, S>(p1, p2);
        } else if constexpr (MU == 2) {
            h[c] = h2_adds<P, -S>(p0, h2_mul_i(p2));
            h[3 + c] = h2_adds<P, S>(p1, h2_mul_i(p3));
        } else {
            h[c] = h2_adds<P, S>(p0, p2);
            h[3 + c] = h2_adds<P, S>(p1, p3);
        }
    }
}

// c + a * b with 16-bit a, b (packed halves selected by the caller) and FP32 c
template <int P>
__device__ __forceinline__ float fma_h(unsigned short a, unsigned short b, float c) {
    float d;
    if constexpr (P == LQ_F16) asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
    else asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
    return d;
}
__device__ __forceinline__ unsigned short lo16(uint32_t w) { return (unsigned short)(w & 0xffffu); }
__device__ __forceinline__ unsigned short hi16(uint32_t w) { return (unsigned short)(w >> 16); }

// uh = U h (ADJ: U^dag h) with U (9 packed complex) and h (6 packed complex) in
// FP16/BF16 and uh in FP32
template <int P, bool ADJ>
__device__ __forceinline__ void su3_mul_h2(const uint32_t (&u)[9], const uint32_t (&h)[6], cplx<float> (&uh)[6]) {
    // copies of h with one part negated: -im (for U h) or -re (for U^dag h)
    uint32_t hn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) hn[k] = h[k] ^ (ADJ ? 0x00008000u : 0x80000000u);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const uint32_t w = ADJ ? u[3 * j + i] : u[3 * i + j];
                const uint32_t x = h[3 * sp + j], xn = hn[3 * sp + j];
                if constexpr (!ADJ) {
                    // (a + ib)(c + id) = ac - bd + i(ad + bc)
                    re = fma_h<P>(lo16(w), lo16(x), re);
                    re = fma_h<P>(hi16(w), hi16(xn), re);
                    im = fma_h<P>(lo16(w), hi16(x), im);
                    im = fma_h<P>(hi16(w), lo16(x), im);
                } else {
                    // (a - ib)(c + id) = ac + bd + i(ad - bc)
                    re = fma_h<P>(lo16(w), lo16(x), re);
                    re = fma_h<P>(hi16(w), hi16(x), re);
                    im = fma_h<P>(lo16(w), hi16(x), im);
                    im = fma_h<P>(hi16(w), lo16(xn), im);
                }
            }
            uh[3 * sp + i] = {re, im};
        }
    }
}

// uh = U h (ADJ: U^dag h), per spin component
template <bool ADJ, typename T>
__device__ __forceinline__ void su3_mul(const cplx<T> (&u)[9], const cplx<T> (&h)[6], cplx<T> (&uh)[6]) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cplx<T> acc = {(T)0, (T)0};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if constexpr (ADJ) cmac_conj(acc, u[3 * j + i], h[3 * sp + j]);
                else cmac(acc, u[3 * i + j], h[3 * sp + j]);
            }
            uh[3 * sp + i] = acc;
        }
    }
}

// Fused |out|^2 of a hop launch: each warp writes one FP64 partial (no block
// barrier, no fence -- the async pipeline of the hop stays undisturbed); a
// separate one-block-per-group launch sums them in a fixed order and sets the
// CG step length (hop_norm_finalize).
__device__ __forceinline__ void hop_norm_warp(double v, double* partial, int warp_index) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) partial[warp_index] = v;
}

}  // namespace lq
