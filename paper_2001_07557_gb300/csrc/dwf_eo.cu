// dwf_eo.cu -- the site-local (5th-dimension) kernels of the domain-wall
// operators: the inverse M5^{-1} of the even-odd preconditioned form, and the
// linear combinations with the shift S that build the Moebius operator.
//
// M5 is the part of D_dw that stays on a 4-d site (Shamir form, walls -mf):
//   (M5 psi)(s) = a psi(s) - P- psi(s+1) - P+ psi(s-1),   a = 5 - M5.
// With gamma_5 = diag(1, 1, -1, -1), P+ keeps spins 0,1 and P- spins 2,3, so M5
// is one real Ls x Ls matrix per chirality, the same for every site, colour
// and spin of that chirality:
//   spins 0,1:  a y(s) - y(s-1),  row 0: a y(0) + mf y(Ls-1)    (lower bidiagonal + corner)
//   spins 2,3:  a y(s) - y(s+1),  row Ls-1: a y(Ls-1) + mf y(0)  (upper bidiagonal + corner)
// and M5^dag swaps the two forms.  Each is B + mf u v^T with B bidiagonal, so
// the inverse is one sweep for B^{-1} plus a Sherman-Morrison correction:
//   z = B^{-1} x (z = (x + z_prev) / a along the sweep),
//   y = z - c w z_end,  w at sweep step j = a^{-(j+1)},  c = mf / (1 + mf a^{-Ls}),
// where z_end is z at the end of the sweep (s = Ls-1 forward, s = 0 backward).
// A thread owns one (site, 16-byte plane) and sweeps twice over the Ls slices:
// once for z_end, once to write y.  Each slice is read before it is written, so
// the call may run in place.  O(Ls) work per component, bandwidth-bound.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "lqcd_kernels.h"
#include "pdl.cuh"

namespace lq {

namespace {

template <typename V, typename T>
__device__ __forceinline__ V axpby4(T a, V x, T b, V y);  // a x + b y

template <>
__device__ __forceinline__ float4 axpby4<float4, float>(float a, float4 x, float b, float4 y) {
    return make_float4(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z), fmaf(a, x.w, b * y.w));
}

template <>
__device__ __forceinline__ double2 axpby4<double2, double>(double a, double2 x, double b, double2 y) {
    return make_double2(fma(a, x.x, b * y.x), fma(a, x.y, b * y.y));
}

// P = LQ_F32: 6 planes of float4 (2 complex) per site; LQ_F64: 12 planes of double2.
// The general site-local matrix alpha + beta S (Shamir M5: alpha = 5 - M5, beta = -1)
// divided by alpha is 1 - g L + corner, g = -beta / alpha: the sweep is
// z(s) = p x(s) + g z(s-1) with p = 1 / alpha, the correction weights w_j = g^(j+1)
// and c = mf / (1 + mf g^Ls).  WITH_B also applies B = b5 + c5 S to the result
// (B commutes with the inverse, both being polynomials in S): S reads the slice
// before s in the sweep's order, and across the wall it reads y at the sweep's
// end, which is y_last = z_end - c g^Ls z_end, known after the first sweep.
template <int P, bool WITH_B>
__global__ void __launch_bounds__(256) m5inv_kernel(char* out, const char* in, int Vh, size_t out_stride,
                                                    size_t in_stride, int Ls, double p_d, double g_d, double c_d,
                                                    double b5_d, double c5_d, double mf_d, int dag) {
    pdl_enter();
    using V = typename std::conditional<P == LQ_F64, double2, float4>::type;
    using T = typename std::conditional<P == LQ_F64, double, float>::type;
    constexpr int NPL = P == LQ_F64 ? 12 : 6;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)Vh * NPL) return;
    const int k = (int)(idx / Vh), i = (int)(idx - (long)k * Vh);  // plane-major: a warp reads 32 sites of a plane
    const bool fwd = (k < NPL / 2) != (dag != 0);  // spins 0,1 sweep upwards in s unless daggered
    const T pc = (T)p_d, g = (T)g_d, c = (T)c_d;
    const char* src = in + ((size_t)k * Vh + i) * sizeof(V);
    char* dst = out + ((size_t)k * Vh + i) * sizeof(V);
    auto slice = [&](int j) { return fwd ? j : Ls - 1 - j; };
    V z = {};
    T w = g;
    for (int j = 0; j < Ls; ++j) {
        const V x = *reinterpret_cast<const V*>(src + (size_t)slice(j) * in_stride);
        z = axpby4<V, T>(pc, x, g, z);
        if (WITH_B && j + 1 < Ls) w *= g;
    }
    const V zend = z;
    V prev = {};
    if constexpr (WITH_B) prev = axpby4<V, T>((T)1, zend, -c * w, zend);  // y at the sweep's last slice
    const T b5 = (T)b5_d, c5 = (T)c5_d;
    T cw = -(T)mf_d * c5;  // S across the wall: -mf
    z = V{};
    w = g;
    for (int j = 0; j < Ls; ++j) {
        const int s = slice(j);
        const V x = *reinterpret_cast<const V*>(src + (size_t)s * in_stride);
        z = axpby4<V, T>(pc, x, g, z);
        const V y = axpby4<V, T>((T)1, z, -c * w, zend);
        if constexpr (WITH_B) {
            *reinterpret_cast<V*>(dst + (size_t)s * out_stride) = axpby4<V, T>(b5, y, cw, prev);
            prev = y;
            cw = c5;
        } else {
            *reinterpret_cast<V*>(dst + (size_t)s * out_stride) = y;
        }
        w *= g;
    }
}

// out(s) = a u(s) + b (S u)(s) + c v(s) + d (S v)(s)   (S^dag for dag; v may be null)
// with S psi(s) = P- psi(s+1) + P+ psi(s-1), walls -mf.  For planes of spins 0,1
// (P+) S reads slice s-1, for spins 2,3 (P-) slice s+1; the dagger swaps them.
// Fields: Ls slices at slice_stride bytes, each nblk parity blocks of Vh sites.
// One thread per (block, plane, site) walks the slices.
template <int P>
__global__ void __launch_bounds__(256) m5_lincomb_kernel(char* out, const char* u, const char* v, int Vh, int nblk,
                                                         size_t slice_stride, int Ls, double a_d, double b_d,
                                                         double c_d, double d_d, double mf_d, int dag) {
    pdl_enter();
    using V = typename std::conditional<P == LQ_F64, double2, float4>::type;
    using T = typename std::conditional<P == LQ_F64, double, float>::type;
    constexpr int NPL = P == LQ_F64 ? 12 : 6;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nblk * NPL * Vh) return;
    const int blk = (int)(idx / ((long)NPL * Vh));
    const int rem = (int)(idx - (long)blk * NPL * Vh);
    const int k = rem / Vh, i = rem - k * Vh;
    const bool down = (k < NPL / 2) != (dag != 0);  // S reads slice s-1 (else s+1)
    const size_t off = (size_t)blk * NPL * Vh * sizeof(V) + ((size_t)k * Vh + i) * sizeof(V);
    const T a = (T)a_d, b = (T)b_d, c = (T)c_d, d = (T)d_d, mf = (T)mf_d;
    auto at = [&](const char* f, int s) { return *reinterpret_cast<const V*>(f + (size_t)s * slice_stride + off); };
    for (int s = 0; s < Ls; ++s) {
        int sn = down ? s - 1 : s + 1;
        T w = 1;
        if (sn < 0) sn = Ls - 1, w = -mf;
        if (sn >= Ls) sn = 0, w = -mf;
        V r = axpby4<V, T>(a, at(u, s), b * w, at(u, sn));
        if (v) r = axpby4<V, T>((T)1, r, (T)1, axpby4<V, T>(c, at(v, s), d * w, at(v, sn)));
        *reinterpret_cast<V*>(out + (size_t)s * slice_stride + off) = r;
    }
}

}  // namespace

cudaError_t launch_m5_lincomb(int prec, void* out, const void* u, const void* v, int Vh, int nblk, size_t slice_stride,
                              int Ls, double a, double b, double c, double d, double mf, bool dag, cudaStream_t st) {
    const int npl = prec == LQ_F64 ? 12 : 6;
    const long n = (long)nblk * npl * Vh;
    const int grid = (int)((n + 255) / 256);
    auto o = static_cast<char*>(out);
    auto pu = static_cast<const char*>(u);
    auto pv = static_cast<const char*>(v);
    if (prec == LQ_F64)
        launch_pdl(m5_lincomb_kernel<LQ_F64>, grid, 256, 0, st, o, pu, pv, Vh, nblk, slice_stride, Ls, a, b, c, d, mf, dag);
    else if (prec == LQ_F32)
        launch_pdl(m5_lincomb_kernel<LQ_F32>, grid, 256, 0, st, o, pu, pv, Vh, nblk, slice_stride, Ls, a, b, c, d, mf, dag);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_m5inv(int prec, void* out, const void* in, int Vh, size_t out_stride, size_t in_stride, int Ls,
                         double M5, double mf, bool dag, cudaStream_t st) {
    const double a = 5.0 - M5;
    double aL = 1.0;  // a^{-Ls}
    for (int s = 0; s < Ls; ++s) aL /= a;
    const double c = mf / (1.0 + mf * aL);
    const int npl = prec == LQ_F64 ? 12 : 6;
    const long n = (long)Vh * npl;
    const int grid = (int)((n + 255) / 256);
    if (prec == LQ_F64)
        launch_pdl(m5inv_kernel<LQ_F64, false>, grid, 256, 0, st, static_cast<char*>(out), static_cast<const char*>(in),
                   Vh, out_stride, in_stride, Ls, 1.0 / a, 1.0 / a, c, 1.0, 0.0, mf, dag);
    else if (prec == LQ_F32)
        launch_pdl(m5inv_kernel<LQ_F32, false>, grid, 256, 0, st, static_cast<char*>(out), static_cast<const char*>(in),
                   Vh, out_stride, in_stride, Ls, 1.0 / a, 1.0 / a, c, 1.0, 0.0, mf, dag);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

bool m5inv_coeffs(double alpha, double beta, double mf, int Ls, double* p, double* g, double* c) {
    if (!(alpha != 0.0) || Ls < 1) return false;
    *p = 1.0 / alpha;
    *g = -beta / alpha;
    double gL = 1.0;
    for (int s = 0; s < Ls; ++s) gL *= *g;
    const double den = 1.0 + mf * gL;
    if (!(den != 0.0) || !std::isfinite(*p) || !std::isfinite(den)) return false;
    *c = mf / den;
    return true;
}

cudaError_t launch_m5inv_general(int prec, void* out, const void* in, int Vh, size_t out_stride, size_t in_stride,
                                 int Ls, double alpha, double beta, double mf, bool with_b, double b5, double c5,
                                 bool dag, cudaStream_t st) {
    double p, g, c;
    if (!m5inv_coeffs(alpha, beta, mf, Ls, &p, &g, &c)) return cudaErrorInvalidValue;
    const int npl = prec == LQ_F64 ? 12 : 6;
    const long n = (long)Vh * npl;
    const int grid = (int)((n + 255) / 256);
    auto o = static_cast<char*>(out);
    auto x = static_cast<const char*>(in);
    if (prec == LQ_F64) {
        if (with_b)
            launch_pdl(m5inv_kernel<LQ_F64, true>, grid, 256, 0, st, o, x, Vh, out_stride, in_stride, Ls, p, g, c, b5, c5,
                       mf, dag);
        else
            launch_pdl(m5inv_kernel<LQ_F64, false>, grid, 256, 0, st, o, x, Vh, out_stride, in_stride, Ls, p, g, c, 1.0,
                       0.0, mf, dag);
    } else if (prec == LQ_F32) {
        if (with_b)
            launch_pdl(m5inv_kernel<LQ_F32, true>, grid, 256, 0, st, o, x, Vh, out_stride, in_stride, Ls, p, g, c, b5, c5,
                       mf, dag);
        else
            launch_pdl(m5inv_kernel<LQ_F32, false>, grid, 256, 0, st, o, x, Vh, out_stride, in_stride, Ls, p, g, c, 1.0,
                       0.0, mf, dag);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lq
