// halo.cu -- building blocks of a time-slab domain decomposition of the Wilson
// operator (one slab of time slices per rank, one ghost slice on each side),
// the counterpart of the MPI shift the paper leaves unfinished (Sec. 3.2):
//   * dslash_apply_slices: the full-lattice hop with output on a range of time
//     slices only, so that the interior of a slab can be computed while its
//     faces are in flight;
//   * lq_face_copy: one time slice of a native field into a slice of another
//     field, times +-1 (the antiperiodic phase at the global time boundary).
// In the native layout, time slice t of a lattice is the run of checkerboard
// sites [t V3/2, (t+1) V3/2) (V3 = L0 L1 L2, even) of every plane of both
// parity blocks, with the same order of sites inside the run.  A face
// therefore moves as contiguous runs.  When the two slice indices differ by an
// odd number, the local parities of the face's sites differ between the two
// lattices, and the copy swaps the parity blocks.
#include <cuda_runtime.h>

#include <cstdint>

#include "handle.h"
#include "pdl.cuh"

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

bool same_space_dims(const lq_handle* a, const lq_handle* b) {
    return a->p.dims[0] == b->p.dims[0] && a->p.dims[1] == b->p.dims[1] && a->p.dims[2] == b->p.dims[2];
}

}  // namespace
}  // namespace lq

using namespace lq;

extern "C" {

int dslash_apply_slices(lq_handle* h, void* out, const void* in, int fmt, int t0, int t1, int dagger, void* stream) {
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

}  // extern "C"
