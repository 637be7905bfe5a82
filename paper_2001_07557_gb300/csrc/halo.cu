// halo.cu -- building blocks of a time-slab domain decomposition of the Wilson
// operator (one slab of time slices per rank, one ghost slice on each side),
// the counterpart of the MPI shift the paper leaves unfinished (Sec. 3.2):
//   * dslash_apply_slices: the full-lattice hop with output on a range of time
//     slices only, so that the interior of a slab can be computed while its
//     faces are in flight;
//   * lq_face_copy: one time slice of a native field into a slice of another
//     field, times +-1 (the antiperiodic phase at the global time boundary);
//   * lq_face_pack / lq_face_unpack: the same exchange with spin-projected
//     faces.  A hop reads a ghost slice only through the time-direction
//     projector (1 + S gamma_t), so only h = psi_up + S psi_dn (2 spins x 3
//     colours, half of the spinor) has to move; the receiver rebuilds a ghost
//     spinor chi with (1 + S gamma_t) chi = (1 + S gamma_t) psi bit for bit.
// In the native layout, time slice t of a lattice is the run of checkerboard
// sites [t V3/2, (t+1) V3/2) (V3 = L0 L1 L2, even) of every plane of both
// parity blocks, with the same order of sites inside the run.  A face
// therefore moves as contiguous runs.  When the two slice indices differ by an
// odd number, the local parities of the face's sites differ between the two
// lattices, and the copy swaps the parity blocks.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "handle.h"
#include "pdl.cuh"
#include "trace.h"

namespace lq {

namespace {

// One 16-byte unit (or norm) of a face per thread.  Units are numbered
// [parity block][plane][site of the run]; FP16/BF16 fields add, per parity
// block, the run of their FP32 site norms, which carry the sign.
template <int P>
__global__ void face_copy_kernel(char* dst, const char* src, int vh_d, int vh_s, int e0_d, int e0_s, int n, int flip,
                                 double scale) {
    pdl_enter();
    constexpr bool NORM = P == LQ_F16 || P == LQ_BF16;
    constexpr int NPL = P == LQ_F64 ? 12 : P == LQ_F32 ? 6 : 3;  // 16-byte planes per site
    const long units = 2L * NPL * n, total = units + (NORM ? 2L * n : 0);
    const long u = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= total) return;
    const size_t site_bytes = NORM ? 52 : 16 * NPL;
    if (u < units) {
        const int p = (int)(u / ((long)NPL * n));
        const int rem = (int)(u - (long)p * NPL * n);
        const int k = rem / n, e = rem - k * n;
        const char* s = src + (size_t)(p ^ flip) * site_bytes * vh_s + ((size_t)k * vh_s + e0_s + e) * 16;
        char* d = dst + (size_t)p * site_bytes * vh_d + ((size_t)k * vh_d + e0_d + e) * 16;
        if constexpr (P == LQ_F64) {
            const double2 v = *reinterpret_cast<const double2*>(s);
            *reinterpret_cast<double2*>(d) = make_double2(scale * v.x, scale * v.y);
        } else if constexpr (P == LQ_F32) {
            const float4 v = *reinterpret_cast<const float4*>(s);
            const float c = (float)scale;
            *reinterpret_cast<float4*>(d) = make_float4(c * v.x, c * v.y, c * v.z, c * v.w);
        } else {
            *reinterpret_cast<uint4*>(d) = *reinterpret_cast<const uint4*>(s);
        }
    } else if constexpr (NORM) {
        const int p = (int)((u - units) / n), e = (int)(u - units - (long)p * n);
        const float* s = reinterpret_cast<const float*>(src + (size_t)(p ^ flip) * site_bytes * vh_s + 48 * (size_t)vh_s);
        float* d = reinterpret_cast<float*>(dst + (size_t)p * site_bytes * vh_d + 48 * (size_t)vh_d);
        d[e0_d + e] = (float)scale * s[e0_s + e];
    }
}

// Spin-projected faces.  In the chiral basis gamma_t = [[0, 1], [1, 0]], so
// (1 + S gamma_t) psi = [h; S h] with h = psi_up + S psi_dn: h[j] = s[j] + S s[6 + j]
// (complex index = spin * 3 + colour), computed with the same additions as the
// hop's own projection.  The wire holds h for the V3/2 sites of each spatial
// parity sp = (x0 + x1 + x2) mod 2, in the slice's run order; the site parity
// block of slice t is sp ^ (t & 1).  Wire planes per spatial-parity block of n
// sites: FP64 6 x 16 B, FP32 3 x 16 B, FP16/BF16 3 x 8 B plus an FP32 norm.
// The ghost gets chi = [h / 2; S h / 2] (FP16/BF16: chi = [h; S h] with the
// norm halved), so the hop's projection of chi, chi_up + S chi_dn, is exactly h.
template <int P>
struct Wire {
    static constexpr bool NORM = P == LQ_F16 || P == LQ_BF16;
    static constexpr int UNIT = NORM ? 8 : 16;           // bytes of one plane element
    static constexpr int NPL = P == LQ_F64 ? 6 : 3;      // planes of h
    static constexpr int SITE = NPL * UNIT + (NORM ? 4 : 0);
};

template <int P, int S>
__global__ void face_pack_kernel(char* wire, const char* src, int vh, int t, int n, double scale) {
    pdl_enter();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= 2 * n) return;
    const int sp = u / n, e = u - sp * n;
    const int p = sp ^ (t & 1);
    const int i = t * n + e;
    char* w = wire + (size_t)sp * Wire<P>::SITE * n;
    if constexpr (P == LQ_F64 || P == LQ_F32) {
        using T = typename std::conditional<P == LQ_F64, double, float>::type;
        cplx<T> s[12];
        load_spinor<P, T>(src + (size_t)p * Prec<P>::spinor_bytes * vh, vh, i, s);
        cplx<T> h[6];
        const T c = (T)scale;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const cplx<T> a = cadds<S>(s[j], s[6 + j]);
            h[j] = {c * a.re, c * a.im};
        }
        if constexpr (P == LQ_F64) {
#pragma unroll
            for (int k = 0; k < 6; ++k) reinterpret_cast<double2*>(w)[(size_t)k * n + e] = make_double2(h[k].re, h[k].im);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                reinterpret_cast<float4*>(w)[(size_t)k * n + e] =
                    make_float4(h[2 * k].re, h[2 * k].im, h[2 * k + 1].re, h[2 * k + 1].im);
        }
    } else {
        const char* blk = src + (size_t)p * Prec<P>::spinor_bytes * vh;
        const uint4* q = reinterpret_cast<const uint4*>(blk);
        uint32_t s[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 v = q[(size_t)k * vh + i];
            s[4 * k] = v.x, s[4 * k + 1] = v.y, s[4 * k + 2] = v.z, s[4 * k + 3] = v.w;
        }
        uint32_t h[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) h[j] = h2_adds<P, S>(s[j], s[6 + j]);
#pragma unroll
        for (int k = 0; k < 3; ++k) reinterpret_cast<uint2*>(w)[(size_t)k * n + e] = make_uint2(h[2 * k], h[2 * k + 1]);
        const float nrm = reinterpret_cast<const float*>(blk + (size_t)48 * vh)[i];
        reinterpret_cast<float*>(w + (size_t)24 * n)[e] = (float)scale * nrm;
    }
}

template <int P, int S>
__global__ void face_unpack_kernel(char* dst, const char* wire, int vh, int t, int n) {
    pdl_enter();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= 2 * n) return;
    const int sp = u / n, e = u - sp * n;
    const int p = sp ^ (t & 1);
    const int i = t * n + e;
    const char* w = wire + (size_t)sp * Wire<P>::SITE * n;
    char* blk = dst + (size_t)p * Prec<P>::spinor_bytes * vh;
    if constexpr (P == LQ_F64 || P == LQ_F32) {
        using T = typename std::conditional<P == LQ_F64, double, float>::type;
        cplx<T> h[6];
        if constexpr (P == LQ_F64) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const double2 v = reinterpret_cast<const double2*>(w)[(size_t)k * n + e];
                h[k] = {v.x, v.y};
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 v = reinterpret_cast<const float4*>(w)[(size_t)k * n + e];
                h[2 * k] = {v.x, v.y};
                h[2 * k + 1] = {v.z, v.w};
            }
        }
        cplx<T> s[12];
        const T half = (T)0.5, sh = (T)(0.5 * S);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            s[j] = {half * h[j].re, half * h[j].im};
            s[6 + j] = {sh * h[j].re, sh * h[j].im};
        }
        store_spinor<P, T>(blk, vh, i, s);
    } else {
        uint32_t s[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 v = reinterpret_cast<const uint2*>(w)[(size_t)k * n + e];
            s[2 * k] = v.x, s[2 * k + 1] = v.y;
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) s[6 + j] = S > 0 ? s[j] : s[j] ^ 0x80008000u;  // S h: flip both sign bits
        uint4* q = reinterpret_cast<uint4*>(blk);
#pragma unroll
        for (int k = 0; k < 3; ++k) q[(size_t)k * vh + i] = make_uint4(s[4 * k], s[4 * k + 1], s[4 * k + 2], s[4 * k + 3]);
        const float nrm = reinterpret_cast<const float*>(w + (size_t)24 * n)[e];
        reinterpret_cast<float*>(blk + (size_t)48 * vh)[i] = 0.5f * nrm;
    }
}

template <int P>
cudaError_t launch_face(bool pack, char* field, char* wire, int vh, int t, int n, int sign, double scale,
                        cudaStream_t st) {
    const int grid = (2 * n + 255) / 256;
    if (pack) {
        const char* src = field;
        if (sign > 0) launch_pdl(face_pack_kernel<P, 1>, grid, 256, 0, st, wire, src, vh, t, n, scale);
        else launch_pdl(face_pack_kernel<P, -1>, grid, 256, 0, st, wire, src, vh, t, n, scale);
    } else {
        const char* w = wire;
        if (sign > 0) launch_pdl(face_unpack_kernel<P, 1>, grid, 256, 0, st, field, w, vh, t, n);
        else launch_pdl(face_unpack_kernel<P, -1>, grid, 256, 0, st, field, w, vh, t, n);
    }
    return cudaGetLastError();
}

size_t wire_bytes(int prec, int n) {
    switch (prec) {
    case LQ_F64: return (size_t)2 * n * Wire<LQ_F64>::SITE;
    case LQ_F32: return (size_t)2 * n * Wire<LQ_F32>::SITE;
    case LQ_F16: return (size_t)2 * n * Wire<LQ_F16>::SITE;
    default: return (size_t)2 * n * Wire<LQ_BF16>::SITE;
    }
}

int face_projected(lq_handle* h, bool pack, void* field, void* wire, int t, int fmt, int sign, double scale,
                   void* stream) {
    if (!h || !field || !wire || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (!(fmt & LQ_NATIVE)) return LQ_ERR_LAYOUT;
    if (sign != 1 && sign != -1) return LQ_ERR_ARG;
    if (t < 0 || t >= h->p.dims[3]) return LQ_ERR_ARG;
    if (!aligned16(field) || !aligned16(wire)) return LQ_ERR_LAYOUT;
    const int prec = fmt & 0xF;
    const int n = h->p.dims[0] * h->p.dims[1] * h->p.dims[2] / 2;
    if (overlap(field, field_bytes(h, fmt, LQ_FULL, 1), wire, wire_bytes(prec, n))) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* f = static_cast<char*>(field);
    char* w = static_cast<char*>(wire);
    const int vh = h->g.Vh;
    cudaError_t e;
    switch (prec) {
    case LQ_F64: e = launch_face<LQ_F64>(pack, f, w, vh, t, n, sign, scale, st); break;
    case LQ_F32: e = launch_face<LQ_F32>(pack, f, w, vh, t, n, sign, scale, st); break;
    case LQ_F16: e = launch_face<LQ_F16>(pack, f, w, vh, t, n, sign, scale, st); break;
    default: e = launch_face<LQ_BF16>(pack, f, w, vh, t, n, sign, scale, st); break;
    }
    return status_of(e);
}

bool same_space_dims(const lq_handle* a, const lq_handle* b) {
    return a->p.dims[0] == b->p.dims[0] && a->p.dims[1] == b->p.dims[1] && a->p.dims[2] == b->p.dims[2];
}

}  // namespace
}  // namespace lq

using namespace lq;

extern "C" {

int dslash_apply_slices(lq_handle* h, void* out, const void* in, int fmt, int t0, int t1, int dagger, void* stream) {
    lq::TraceRange trace_("lqcd/dslash_slices");
    if (!h || !out || !in || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (!(fmt & LQ_NATIVE)) return LQ_ERR_LAYOUT;
    if (t0 < 0 || t1 > h->p.dims[3] || t0 >= t1) return LQ_ERR_ARG;
    if (!aligned16(out) || !aligned16(in)) return LQ_ERR_LAYOUT;
    const size_t nb = field_bytes(h, fmt, LQ_FULL, 1);
    if (overlap(out, nb, in, nb)) return LQ_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int prec = fmt & 0xF;
    const int vh3 = h->p.dims[0] * h->p.dims[1] * h->p.dims[2] / 2;  // sites of one parity in a time slice
    HopArgs a;
    int rc = prep_wilson_full(h, prec, static_cast<char*>(out), static_cast<const char*>(in), 1, &a, st);
    if (rc) return rc;
    a.site0 = t0 * vh3;
    a.nsite = (t1 - t0) * vh3;
    a.red_partial = nullptr;  // a partial hop carries no fused norm
    a.red_st = nullptr;
    return status_of(launch_hop(prec, a, link_r12(h, prec), dagger != 0, EPI_DIAG, h->hop_block[prec], st));
}

int lq_face_copy(lq_handle* hd, void* dst, int t_dst, lq_handle* hs, const void* src, int t_src, int fmt,
                 double scale, void* stream) {
    lq::TraceRange trace_("lqcd/face_copy");
    if (!hd || !hs || !dst || !src || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (!(fmt & LQ_NATIVE)) return LQ_ERR_LAYOUT;
    if (!same_space_dims(hd, hs)) return LQ_ERR_ARG;
    if (t_dst < 0 || t_dst >= hd->p.dims[3] || t_src < 0 || t_src >= hs->p.dims[3]) return LQ_ERR_ARG;
    if (!aligned16(dst) || !aligned16(src)) return LQ_ERR_LAYOUT;
    if (dst == src && t_dst == t_src) return LQ_ERR_ARG;  // a slice onto itself
    DeviceGuard dg(hd->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int prec = fmt & 0xF;
    const int vh3 = hd->p.dims[0] * hd->p.dims[1] * hd->p.dims[2] / 2;
    const int npl = prec == LQ_F64 ? 12 : prec == LQ_F32 ? 6 : 3;
    const long total = 2L * npl * vh3 + ((prec == LQ_F16 || prec == LQ_BF16) ? 2L * vh3 : 0);
    const int grid = (int)((total + 255) / 256);
    char* d = static_cast<char*>(dst);
    const char* s = static_cast<const char*>(src);
    const int vd = hd->g.Vh, vs = hs->g.Vh, e0d = t_dst * vh3, e0s = t_src * vh3, flip = (t_dst - t_src) & 1;
    switch (prec) {
    case LQ_F64: launch_pdl(face_copy_kernel<LQ_F64>, grid, 256, 0, st, d, s, vd, vs, e0d, e0s, vh3, flip, scale); break;
    case LQ_F32: launch_pdl(face_copy_kernel<LQ_F32>, grid, 256, 0, st, d, s, vd, vs, e0d, e0s, vh3, flip, scale); break;
    case LQ_F16: launch_pdl(face_copy_kernel<LQ_F16>, grid, 256, 0, st, d, s, vd, vs, e0d, e0s, vh3, flip, scale); break;
    default: launch_pdl(face_copy_kernel<LQ_BF16>, grid, 256, 0, st, d, s, vd, vs, e0d, e0s, vh3, flip, scale); break;
    }
    return status_of(cudaGetLastError());
}

int lq_face_wire_bytes(const lq_handle* h, int fmt, size_t* bytes) {
    if (!h || !bytes || !valid_fmt(fmt)) return LQ_ERR_ARG;
    *bytes = wire_bytes(fmt & 0xF, h->p.dims[0] * h->p.dims[1] * h->p.dims[2] / 2);
    return LQ_OK;
}

int lq_face_pack(lq_handle* h, void* wire, const void* src, int t_src, int fmt, int sign, double scale, void* stream) {
    lq::TraceRange trace_("lqcd/face_pack");
    return face_projected(h, true, const_cast<void*>(src), wire, t_src, fmt, sign, scale, stream);
}

int lq_face_unpack(lq_handle* h, void* dst, int t_dst, const void* wire, int fmt, int sign, void* stream) {
    lq::TraceRange trace_("lqcd/face_unpack");
    return face_projected(h, false, dst, const_cast<void*>(wire), t_dst, fmt, sign, 1.0, stream);
}

}  // extern "C"
