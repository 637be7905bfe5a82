// hop.cuh -- the Wilson hopping kernel (one thread per output site) and its
// epilogues.  Included by one translation unit per storage precision.
//
// For output parity p the kernel computes, per site x of parity p,
//   out(x) = c_hop * (H psi)(x) + c_diag * x_in(x) [+ 5th-dimension terms]
// where psi is the parity 1-p field.  The 8 neighbours are gathered from the
// native structure-of-arrays blocks (16-byte vector loads, consecutive
// threads on consecutive sites), spin-projected to half spinors, multiplied
// by U or U^dag in registers, reconstructed and accumulated (Sec. 3.1 of the
// paper builds the same stencil from shifts of whole SIMD arrays; here the
// shift is a per-thread neighbour index).
#pragma once

#include "lqcd_internal.cuh"
#include "lqcd_kernels.h"
#include "pdl.cuh"

namespace lq {

template <int P, bool R12, bool DAG, int EPI, bool RED>
__global__ void __launch_bounds__(128) wilson_hop_kernel(const HopArgs a) {
    pdl_enter();
    using T = typename Prec<P>::real;
    // grid.x = (rhs, output parity, site tile), rhs fastest: the right-hand sides, or
    // 5th-dimension slices, of one site tile run together and share each link through
    // L2/L1, and so do the two parities of a tile (one parity's outputs read the other's
    // block as neighbours, its own as the diagonal / 5th-dimension input)
    const int rhs = blockIdx.x % a.nrhs;
    const int pt = blockIdx.x / a.nrhs;  // parity x tile index
    const Geom& g = a.g;
    const int end = a.nsite ? a.site0 + a.nsite : g.Vh;
    const int i0 = a.site0 + (pt / a.nparity) * blockDim.x + threadIdx.x;
    const bool active = i0 < end;
    if constexpr (!RED) {
        if (!active) return;
    }
    const int i = active ? i0 : end - 1;  // (fused norm: a thread past the end stores nothing)
    const int p = a.parity0 + pt % a.nparity;
    if (a.skip && a.skip[(EPI == EPI_DWF ? 0 : rhs) * a.skip_stride]) return;

    const char* __restrict__ in = a.in[p] + (size_t)rhs * a.in_rhs;
    int x[4];
    cb_coords(g, i, p, x);

    // forward (x+mu) and backward (x-mu) checkerboard indices and phases
    const int xh = x[0] >> 1;
    int nf[4], nb[4];
    bool sf[4], sb[4];
    {
        int xf = x[0] + 1, xb = x[0] - 1;
        sf[0] = (xf == g.L[0]);
        sb[0] = (xb < 0);
        if (sf[0]) xf = 0;
        if (sb[0]) xb = g.L[0] - 1;
        nf[0] = i - xh + (xf >> 1);
        nb[0] = i - xh + (xb >> 1);
        int step = g.Lh0;
#pragma unroll
        for (int mu = 1; mu < 4; ++mu) {
            const bool top = (x[mu] == g.L[mu] - 1), bot = (x[mu] == 0);
            sf[mu] = top;
            sb[mu] = bot;
            nf[mu] = top ? i - (g.L[mu] - 1) * step : i + step;
            nb[mu] = bot ? i + (g.L[mu] - 1) * step : i - step;
            step *= g.L[mu];
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            sf[mu] = sf[mu] && (g.bc[mu] < 0);
            sb[mu] = sb[mu] && (g.bc[mu] < 0);
            nf[mu] = check_site(nf[mu], g.Vh);
            nb[mu] = check_site(nb[mu], g.Vh);
        }
    }

    cplx<T> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {(T)0, (T)0};

    // forward: (1 - gamma) U_mu(x) psi(x+mu); dagger: (1 + gamma)
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const char* __restrict__ Lp = a.links + (size_t)(p * 4) * a.link_block;
    const char* __restrict__ Lq = a.links + (size_t)((1 - p) * 4) * a.link_block;

    // The 8 directions D = 2 mu + (0 forward, 1 backward) run as a two-stage
    // pipeline: the packed spinor and link of direction D+1 are loaded before
    // direction D is unpacked and computed.  FP16/BF16: the site norm and the
    // boundary phase multiply the accumulation FMAs; FP32/FP64: a crossing hop
    // negates its half spinor.
    constexpr bool NORM = Prec<P>::has_norm;
    RawSpinor<P> rs[2];
    RawLink<P, R12> rl[2];
    auto load_dir = [&](int D, int slot) {
        const int mu = D >> 1;
        const bool fwd = (D & 1) == 0;
        raw_load(rs[slot], in, g.Vh, fwd ? nf[mu] : nb[mu]);
        raw_load(rl[slot], (fwd ? Lp : Lq) + (size_t)mu * a.link_block, g.Vh, fwd ? i : nb[mu]);
    };
#define LQ_HOP_DIR(D)                                                                  \
    {                                                                                  \
        constexpr int MU = (D) >> 1;                                                   \
        constexpr bool FWD = ((D)&1) == 0;                                             \
        constexpr int S = FWD ? SF : SB;                                               \
        if constexpr ((D) < 7) load_dir((D) + 1, ((D) + 1) & 1);                      \
        cplx<T> s[12], h[6], uh[6], u[9];                                              \
        T nrm;                                                                         \
        raw_unpack<P, T>(rs[(D)&1], s, nrm);                                           \
        project<MU, S>(s, h);                                                          \
        raw_unpack<P, R12, T>(rl[(D)&1], u);                                           \
        const bool sgn = FWD ? sf[MU] : sb[MU];                                        \
        if constexpr (NORM) {                                                          \
            su3_mul<!FWD>(u, h, uh);                                                   \
            reconstruct_fma<MU, S>(acc, uh, sgn ? -nrm : nrm);                         \
        } else {                                                                       \
            if (sgn) {                                                                 \
                _Pragma("unroll") for (int k = 0; k < 6; ++k) h[k] = cneg(h[k]);       \
            }                                                                          \
            su3_mul<!FWD>(u, h, uh);                                                   \
            reconstruct_add<MU, S>(acc, uh);                                           \
        }                                                                              \
    }
    load_dir(0, 0);
    LQ_HOP_DIR(0)
    LQ_HOP_DIR(1)
    LQ_HOP_DIR(2)
    LQ_HOP_DIR(3)
    LQ_HOP_DIR(4)
    LQ_HOP_DIR(5)
    LQ_HOP_DIR(6)
    LQ_HOP_DIR(7)
#undef LQ_HOP_DIR

    const T ch = (T)a.c_hop;
    cplx<T> o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = {ch * acc[k].re, ch * acc[k].im};

    if constexpr (EPI >= EPI_DIAG) {
        const T cd = (T)a.c_diag;
        const char* __restrict__ xb = a.x[p] + (size_t)rhs * a.x_rhs;
        cplx<T> xs[12];
        load_spinor<P, T>(xb, g.Vh, i, xs);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            o[k].re = fma(cd, xs[k].re, o[k].re);
            o[k].im = fma(cd, xs[k].im, o[k].im);
        }
    }
    if constexpr (EPI == EPI_DWF) {
        // P+ = upper spins (gamma_5 = diag(1,1,-1,-1)).  Non-dagger: upper from
        // s-1, lower from s+1; dagger swaps.  Coefficient c_shift (Shamir: -1), times -mf across the wall.
        const int Ls = a.Ls;
        const int s = rhs;
        const int s_up = DAG ? (s + 1 == Ls ? 0 : s + 1) : (s == 0 ? Ls - 1 : s - 1);
        const int s_dn = DAG ? (s == 0 ? Ls - 1 : s - 1) : (s + 1 == Ls ? 0 : s + 1);
        const bool wrap_up = DAG ? (s + 1 == Ls) : (s == 0);
        const bool wrap_dn = DAG ? (s == 0) : (s + 1 == Ls);
        const T c_up = wrap_up ? (T)(-a.c_shift * a.mf) : (T)a.c_shift;
        const T c_dn = wrap_dn ? (T)(-a.c_shift * a.mf) : (T)a.c_shift;
        cplx<T> su[12], sd[12];
        load_spinor<P, T>(a.x[p] + (size_t)s_up * a.x_rhs, g.Vh, i, su);
        load_spinor<P, T>(a.x[p] + (size_t)s_dn * a.x_rhs, g.Vh, i, sd);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            o[k].re = fma(c_up, su[k].re, o[k].re);
            o[k].im = fma(c_up, su[k].im, o[k].im);
            o[6 + k].re = fma(c_dn, sd[6 + k].re, o[6 + k].re);
            o[6 + k].im = fma(c_dn, sd[6 + k].im, o[6 + k].im);
        }
    }
    if (active) store_spinor<P, T>(a.out[p] + (size_t)rhs * a.out_rhs, g.Vh, i, o);
    if constexpr (RED) {
        double v = 0;
        if (active) {
#pragma unroll
            for (int k = 0; k < 12; ++k) v += (double)(o[k].re * o[k].re + o[k].im * o[k].im);
        }
        // warp partials, group-major: [group][warp of the group's blocks]
        const int wpb = blockDim.x >> 5;
        const int grp = EPI == EPI_DWF ? 0 : rhs;
        const int nblk = EPI == EPI_DWF ? gridDim.x : gridDim.x / a.nrhs;
        const int bidx = EPI == EPI_DWF ? blockIdx.x : pt;
        hop_norm_warp(v, a.red_partial + (size_t)grp * nblk * wpb, bidx * wpb + (threadIdx.x >> 5));
    }
}

template <int P>
cudaError_t launch_hop_prec(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    const int nsite = a.nsite ? a.nsite : a.g.Vh;
    dim3 grid(((nsite + block - 1) / block) * a.nrhs * a.nparity);
    dim3 blk(block);
    const bool red = a.red_partial != nullptr;
    if (red && epi == EPI_HOP) return cudaErrorInvalidValue;
#define LQ_LAUNCH(R, D, E, RD) launch_pdl(wilson_hop_kernel<P, R, D, E, RD>, grid, blk, 0, st, a)
#define LQ_EPI(R, D)                                                                           \
    switch (epi) {                                                                             \
    case EPI_HOP: LQ_LAUNCH(R, D, EPI_HOP, false); break;                                      \
    case EPI_DIAG: if (red) LQ_LAUNCH(R, D, EPI_DIAG, true); else LQ_LAUNCH(R, D, EPI_DIAG, false); break; \
    default: if (red) LQ_LAUNCH(R, D, EPI_DWF, true); else LQ_LAUNCH(R, D, EPI_DWF, false); break;         \
    }
    if (r12) {
        if (dag) { LQ_EPI(true, true) } else { LQ_EPI(true, false) }
    } else {
        if (dag) { LQ_EPI(false, true) } else { LQ_EPI(false, false) }
    }
#undef LQ_EPI
#undef LQ_LAUNCH
    return cudaGetLastError();
}

}  // namespace lq
