// blas.h -- solver vector kernels: descriptors and launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "lqcd_internal.cuh"

namespace lq {

// A native field of nrhs right-hand sides; each rhs is nblk parity blocks of
// Vh sites (1 for a half field, 2 for a full field, 2*Ls for a 5-d field),
// rhs_stride bytes apart.
struct VecRef {
    char* ptr;
    int prec;
    size_t rhs_stride;
};

struct Scratch {
    double* partial;    // reduce_scratch_doubles() entries
    unsigned* tickets;  // one per rhs, zero before the first launch (each launch leaves them zero)
};

enum { FIN_STORE = 0, FIN_ALPHA = 1 };

size_t reduce_scratch_doubles(int Vh, int nblk, int nrhs);

// One (lattice, right-hand side) segment of a batched CG over lattices of
// different sizes: base pointers of its x, p, r, q vectors (nblk parity blocks
// of Vh sites each), its scalars, and its reduction partials (gx) and ticket.
struct BSeg {
    char* x;
    char* p;
    char* r;
    char* q;
    int Vh;
    int nblk;
    CgScalars* st;
    double* partial;
    unsigned* ticket;
};

// Batched CG steps over nseg segments, gx blocks per segment (grid = gx x nseg).
cudaError_t launch_bdot_alpha(const BSeg* segs, int nseg, int gx, int pp, cudaStream_t s);
cudaError_t launch_bupdate(const BSeg* segs, int nseg, int gx, int px, int pp, cudaStream_t s);
cudaError_t launch_bxpay(const BSeg* segs, int nseg, int gx, int pp, int pr, cudaStream_t s);

cudaError_t launch_dot(const VecRef& a, const VecRef& b, int Vh, int nblk, int nrhs, const Scratch& sc,
                       CgScalars* st, double* out, int fin, cudaStream_t s);
cudaError_t launch_cg_update(const VecRef& x, const VecRef& p, const VecRef& r, const VecRef& q, int Vh, int nblk,
                             int nrhs, const Scratch& sc, CgScalars* st, cudaStream_t s);
cudaError_t launch_cg_xpay(const VecRef& p, const VecRef& r, int Vh, int nblk, int nrhs, const CgScalars* st,
                           cudaStream_t s);
cudaError_t launch_axpby(const VecRef& y, const VecRef& x, double a, double b, int Vh, int nblk, int nrhs,
                         cudaStream_t s);
// Sum the warp partials of the last fused-norm hop (ngroups groups of nwarps
// each) in a fixed order and set pAp and alpha of each group.  The second level
// of the sum uses sc (scratch entries per group as for vectors of Vh x nblk sites).
cudaError_t launch_hop_norm_finalize(const double* partial, int nwarps, int ngroups, CgScalars* st,
                                     const Scratch& sc, int Vh, int nblk, cudaStream_t s);
// Complex dot <a, b> per rhs of nsites sites each (site-major or native fmt);
// scratch: 2 * kMaxGrid * nrhs doubles, tickets: nrhs zeros; result: 2 * nrhs doubles (device).
constexpr int kMaxGrid = 152 * 8;
cudaError_t launch_cdot(int fmt, const void* a, const void* b, size_t rhs_stride, long nsites, int Vh, int nrhs,
                        double* scratch, unsigned* tickets, double* result, cudaStream_t s);

cudaError_t launch_cg_init(CgScalars* st, const double* rr, const double* bb, double tol, int maxiter, int nrhs,
                           cudaStream_t s);

}  // namespace lq
