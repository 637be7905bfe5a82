// lqcd_kernels.h -- host-side interface between the C ABI layer and the
// kernels (launch descriptors and launcher declarations).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "lqcd_internal.cuh"

namespace lq {

enum { EPI_HOP = 0, EPI_DIAG = 1, EPI_DWF = 2 };

// One hop launch.  Pointers are indexed by OUTPUT parity p: in[p] is the
// parity 1-p input block of rhs 0, out[p] / x[p] the parity-p blocks of rhs 0.
// Consecutive rhs (or 5th-dimension slices) are *_rhs bytes apart.
struct HopArgs {
    const char* links;  // native links of the launch precision: [parity][mu] blocks
    size_t link_block;  // bytes of one (parity, mu) block
    Geom g;
    const char* in[2];
    char* out[2];
    const char* x[2];
    size_t in_rhs, out_rhs, x_rhs;
    int parity0;  // first output parity
    int nparity;  // 1 (one parity) or 2 (both: full-lattice operator)
    int site0, nsite;  // output checkerboard sites [site0, site0 + nsite) of each parity (nsite 0: all Vh)
    int nrhs;     // right-hand sides, or Ls for the domain-wall epilogue
    double c_hop, c_diag;
    int Ls;
    double mf;
    // domain-wall epilogue: coefficient of (S x)(s) = P+ x(s_up) + P- x(s_dn), walls
    // -mf (the Shamir operator's site-local part takes -1; set at every EPI_DWF launch)
    double c_shift;
    // 1: a launch of at least 8 right-hand sides in FP16/BF16 with 18-real links runs
    // its SU(3) products on the tensor cores (hop_mma.cuh); 0: CUDA cores only
    int mma;
    const int* skip;  // optional per-rhs flags (skip[rhs * skip_stride]): a set flag ends the block at once
    int skip_stride;
    // optional fused |out|^2 per right-hand side (one group for the domain wall):
    // one FP64 partial per warp; hop_norm_finalize sums them and sets
    // st.pAp = |out|^2 = <p, K^dag K p> and st.alpha = st.rr / st.pAp
    double* red_partial;
    unsigned* red_ticket;  // unused by the hop (kept for the layout of callers)
    CgScalars* red_st;
    // persistent batch hop only: 128-site tiles per work item of this lattice (its autotuned size)
    int batch_mult;
};

// Every hop launch uses blocks of this many threads (the fused-norm partial
// count depends on it).
constexpr int kHopThreads = 128;

// Warp partials per reduction group of a fused-norm hop launch over nparity
// parities and `slices` 5th-dimension slices (1 for Wilson).
inline size_t hop_red_warps(int Vh, int nparity, int slices) {
    return (size_t)((Vh + kHopThreads - 1) / kHopThreads) * (kHopThreads / 32) * nparity * slices;
}


cudaError_t launch_hop(int prec, const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st);

// out = M5^{-1} in (dag: (M5^dag)^{-1}) on the Ls slices of one parity block of
// a native FP64/FP32 5-d field; slice s of out/in at s * out_stride/in_stride
// bytes.  In place allowed.  (dwf_eo.cu)
cudaError_t launch_m5inv(int prec, void* out, const void* in, int Vh, size_t out_stride, size_t in_stride, int Ls,
                         double M5, double mf, bool dag, cudaStream_t st);

// The general site-local inverse (alpha + beta S)^{-1} (dag: with S^dag), times
// B = b5 + c5 S (or S^dag) when with_b.  Same layouts as launch_m5inv; in place
// allowed.  m5inv_coeffs gives false when the matrix is singular (alpha = 0 or
// 1 + mf (-beta/alpha)^Ls = 0); the launcher then returns cudaErrorInvalidValue
// without launching.  (dwf_eo.cu)
bool m5inv_coeffs(double alpha, double beta, double mf, int Ls, double* p, double* g, double* c);
cudaError_t launch_m5inv_general(int prec, void* out, const void* in, int Vh, size_t out_stride, size_t in_stride,
                                 int Ls, double alpha, double beta, double mf, bool with_b, double b5, double c5,
                                 bool dag, cudaStream_t st);

// out(s) = a u(s) + b (S u)(s) + c v(s) + d (S v)(s), S psi(s) = P- psi(s+1) +
// P+ psi(s-1) with walls -mf (dag: S^dag); v may be null.  Native FP64/FP32
// 5-d fields: Ls slices at slice_stride bytes of nblk parity blocks.  out must
// not overlap u or v.  (dwf_eo.cu)
cudaError_t launch_m5_lincomb(int prec, void* out, const void* u, const void* v, int Vh, int nblk, size_t slice_stride,
                              int Ls, double a, double b, double c, double d, double mf, bool dag, cudaStream_t st);
// index-checked build: out-of-range indices counted by the hop translation units
// since the last read (cleared by the read); ~0 on a CUDA error
unsigned long long index_faults_f64(long long* first);
unsigned long long index_faults_f32(long long* first);
unsigned long long index_faults_f16(long long* first);
unsigned long long index_faults_bf16(long long* first);
cudaError_t launch_hop_f64(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st);
cudaError_t launch_hop_f32(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st);
cudaError_t launch_hop_f16(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st);
cudaError_t launch_hop_bf16(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st);

// Persistent hop over a batch of lattices (FP32 / FP16 / BF16 storage):
// args[nlat] device launch descriptors, lat_off[nlat + 1] device prefix sums
// of each lattice's work items (ceil(Vh / (128 args[l].batch_mult)) x nrhs x
// nparity).  grid == 0: *occ receives the resident blocks per SM (nothing is
// launched).
cudaError_t launch_hop_batch(int prec, const HopArgs* args, const int* lat_off, int nlat, bool r12, bool dag, int epi,
                             int grid, cudaStream_t st, int* occ);
cudaError_t launch_hop_batch_f32(const HopArgs*, const int*, int, bool, bool, int, int, cudaStream_t, int*);
cudaError_t launch_hop_batch_f16(const HopArgs*, const int*, int, bool, bool, int, int, cudaStream_t, int*);
cudaError_t launch_hop_batch_bf16(const HopArgs*, const int*, int, bool, bool, int, int, cudaStream_t, int*);

// ----------------------------------------------------------- conversions
// Spinor fields.  "site-major" = [rhs][site][4][3][2] in F64/F32, sites either
// the full lattice in lexicographic order (full = true) or one parity in cb
// order (full = false).  Native = [rhs][parity][planes] (full) or [rhs][planes].
cudaError_t launch_spinor_to_native(int dst_prec, void* dst, int src_prec, const void* src, const Geom& g,
                                    bool full, int parity, int nrhs, cudaStream_t st);
cudaError_t launch_spinor_from_native(int dst_prec, void* dst, int src_prec, const void* src, const Geom& g,
                                      bool full, int parity, int nrhs, cudaStream_t st);
cudaError_t launch_native_convert(int dst_prec, void* dst, int src_prec, const void* src, int Vh, int nblocks,
                                  cudaStream_t st);
// Largest deviation from SU(3) of nlinks site-major 3x3 links (max |U^dag U - 1|
// entry and |det U - 1|; +inf for a NaN); synchronises st.
cudaError_t link_su3_deviation(int src_prec, const void* src, long nlinks, double* dev, cudaStream_t st);
// Gauge links: site-major [site][mu][3][3][2] (F64/F32) -> native [parity][mu] blocks.
cudaError_t launch_links_to_native(int dst_prec, bool r12, void* dst, int src_prec, const void* src, const Geom& g,
                                   cudaStream_t st);

}  // namespace lq
