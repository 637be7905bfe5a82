// hop_shared.cuh -- the Wilson hop of a launch with several right-hand sides
// (or domain-wall slices) that share each link, for FP32 storage.
//
// In the one-right-hand-side kernel (hop_async.cuh) every block streams the
// 8 links of its sites through L2, so a launch of N right-hand sides fetches
// every link N times from L2 and recomputes the neighbour indices N times.
// Here a block owns a tile of kShSites sites of one parity and ALL the
// right-hand sides of the launch:
//   * threads (s, g): site s of the tile, group g of G; group g takes the
//     right-hand sides g, g + G, g + 2G, ... one after another;
//   * the block stages the tile's 8 links per site into shared memory once
//     (one cp.async per 16-byte chunk, spread over the groups), then a
//     barrier; every later use of a link by any right-hand side reads it
//     from there;
//   * each thread streams its neighbour spinors through a private S-stage
//     ring of cp.async copies as in hop_async.cuh; the ring runs on across
//     the right-hand sides of the thread, so the copies of the next
//     right-hand side's first directions overlap the last ones of the
//     current one, and the first ones overlap the staging of the links.
// Per site and right-hand side the L2 traffic drops from 8 neighbours + 8
// links to 8 neighbours + 8/N links (24^3 x 48, 12 right-hand sides, FP32:
// 14.1 -> 8.8 GB per launch).  Measured, FP16/BF16 storage (whose hops are
// issue-bound) do not gain from it and keep the hop_async.cuh kernel.
// The arithmetic per site and right-hand side is that of hop_async.cuh, in the
// same order, so a right-hand side comes out bit for bit as it does from a
// launch of its own; the fused-norm partials fill the same slots with the same
// warp sums.
#pragma once

#include <cuda_pipeline.h>

#include "hop_async.cuh"

namespace lq {

// Block shape, measured on 24^3 x 48 with 12 right-hand sides (FP32) and on the
// 16^4 x 16 domain wall: 32 sites x 4 groups with five resident blocks of 128
// threads (102 registers, 43 KB of shared memory each) 494 / 72 us; 64 x 4 with
// two blocks of 256 threads (128 registers) 527 / 76 us; 64 x 3 with three
// blocks 533 / 86 us; 32 x 8 with three blocks 606 / 84 us.
constexpr int kShSites = 32;     // sites per tile (one warp of each group)
constexpr int kShGroups = 4;     // groups of threads per block, each taking every kShGroups-th right-hand side
constexpr int kShMinBlocks = 5;  // resident blocks per SM the register budget is set for

// The tile's links in shared memory: per direction, LinkLayout's 16-byte
// chunks chunk-major over the tile's sites, then the tail chunk.
template <int P, bool R12>
struct LinkTile {
    using LL = LinkLayout<P, R12>;
    static constexpr int NS = kShSites;
    static constexpr int DIR = (LL::NFULL * 16 + LL::TAIL) * NS;
    static constexpr int BYTES = 8 * DIR;
};

template <int P, bool R12>
__device__ __forceinline__ void tile_link_stage(unsigned char* dir, const char* __restrict__ blk, int Vh, int site,
                                                int s) {
    using LL = LinkLayout<P, R12>;
    constexpr int NS = kShSites;
#pragma unroll
    for (int c = 0; c < LL::NFULL; ++c)
        __pipeline_memcpy_async(dir + (c * NS + s) * 16, blk + ((size_t)c * Vh + site) * 16, 16);
    if constexpr (LL::TAIL > 0)
        __pipeline_memcpy_async(dir + LL::NFULL * 16 * NS + s * LL::TAIL,
                                blk + (size_t)LL::NFULL * 16 * Vh + (size_t)site * LL::TAIL, LL::TAIL);
}

template <int P, bool R12>
__device__ __forceinline__ void tile_link(const unsigned char* dir, int s, cplx<float> (&u)[9]) {
    using LL = LinkLayout<P, R12>;
    constexpr int NS = kShSites;
    RawLink<P, R12> r;
#pragma unroll
    for (int c = 0; c < LL::NFULL; ++c) {
        const uint4 v = *reinterpret_cast<const uint4*>(dir + (c * NS + s) * 16);
        r.w[4 * c] = v.x;
        r.w[4 * c + 1] = v.y;
        r.w[4 * c + 2] = v.z;
        r.w[4 * c + 3] = v.w;
    }
    const unsigned char* tail = dir + LL::NFULL * 16 * NS;
    if constexpr (LL::TAIL == 8) {
        const uint2 v = *reinterpret_cast<const uint2*>(tail + s * 8);
        r.w[4 * LL::NFULL] = v.x;
        r.w[4 * LL::NFULL + 1] = v.y;
    } else if constexpr (LL::TAIL == 4) {
        r.w[4 * LL::NFULL] = *reinterpret_cast<const uint32_t*>(tail + s * 4);
    }
    raw_unpack<P, R12, float>(r, u);
}

template <int P, bool R12, int NT, int S>
constexpr int shared_smem_bytes() {
    return LinkTile<P, R12>::BYTES + S * AsyncStage<P, R12, NT>::SPIN_BYTES;
}

// Slot of the fused-norm partial of the warp covering 32-site chunk c32 of a
// parity block: the slot hop_async.cuh's 128-thread blocks give the same
// sites (warp c32 % 4 of tile c32 / 4), so one finalize serves both kernels.
__device__ __forceinline__ size_t shared_red_slot(const HopArgs& a, int epi_dwf, int rhs, int pidx, int c32) {
    const int tiles128 = (a.g.Vh + kHopThreads - 1) / kHopThreads;
    const int w4 = c32 & 3, t128 = c32 >> 2;
    if (epi_dwf) return ((size_t)(t128 * a.nparity + pidx) * a.nrhs + rhs) * 4 + w4;
    return (size_t)rhs * tiles128 * a.nparity * 4 + (size_t)(t128 * a.nparity + pidx) * 4 + w4;
}

template <int P, bool R12, bool DAG, int EPI, int G, int S, bool RED>
__global__ void __launch_bounds__(kShSites* G, kShMinBlocks) wilson_hop_shared_kernel(const HopArgs a) {
    static_assert(!Prec<P>::has_norm, "the shared-link hop serves FP32 storage");
    static_assert(kShSites % 32 == 0, "a warp must hold sites of one group (one right-hand side)");
    constexpr int NS = kShSites, NT = NS * G;
    using T = float;
    using St = AsyncStage<P, R12, NT>;
    using LT = LinkTile<P, R12>;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* links = smem;             // LT::BYTES
    unsigned char* ring = smem + LT::BYTES;  // S stages of St::SPIN_BYTES
    const int t = threadIdx.x;
    const int s = t % NS, grp = t / NS;
    // grid.x = (output parity, tile), parity fastest: the two parities of a tile run
    // together (one parity's outputs read the other's block as neighbours, its own as
    // the diagonal / 5th-dimension input)
    const int pidx = blockIdx.x % a.nparity;
    const int tile = blockIdx.x / a.nparity;
    const Geom& g = a.g;
    const int i0 = tile * NS + s;
    const bool active = i0 < g.Vh;
    const int i = active ? i0 : g.Vh - 1;  // a thread past the end recomputes the last site, stores nothing
    const int p = a.parity0 + pidx;
    pdl_enter();  // every global access of the block comes after this (programmatic dependent launch)
    if (EPI == EPI_DWF && a.skip && a.skip[0]) return;  // one flag for the whole 5-d system, uniform per block
    // this thread's right-hand sides: grp, grp + G, ... (bit k: grp + k G), minus the finished ones
    unsigned mask = 0;
    for (int k = 0; grp + k * G < a.nrhs; ++k)
        if (EPI == EPI_DWF || !a.skip || !a.skip[(grp + k * G) * a.skip_stride]) mask |= 1u << k;

    int x[4];
    cb_coords(g, i, p, x);
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
    const char* __restrict__ Lp = a.links + (size_t)(p * 4) * a.link_block;
    const char* __restrict__ Lq = a.links + (size_t)((1 - p) * 4) * a.link_block;

    // the tile's links, staged once: group g copies directions g, g + G, ...
    for (int D = grp; D < 8; D += G) {
        const int mu = D >> 1;
        const bool fwd = (D & 1) == 0;
        tile_link_stage<P, R12>(links + D * LT::DIR, (fwd ? Lp : Lq) + (size_t)mu * a.link_block, g.Vh,
                                fwd ? i : nb[mu], s);
    }
    __pipeline_commit();

    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;

    // ring of neighbour spinors; item n = (n / 8)-th right-hand side of the thread, direction n % 8
    int cur = mask ? __ffs(mask) - 1 : 0;  // index k of the current right-hand side
    unsigned rest = mask & (mask - 1);
    auto in_of = [&](int k) { return a.in[p] + (size_t)(grp + k * G) * a.in_rhs; };
    auto issue = [&](int k, int D, int slot) {
        const int mu = D >> 1;
        const bool fwd = (D & 1) == 0;
        async_spinor<P, R12, NT>(ring + slot * St::SPIN_BYTES, in_of(k), g.Vh, fwd ? nf[mu] : nb[mu], t);
    };
    // prologue: items 0 .. S-2 (directions of the first right-hand side), in flight
    // together with the link copies; then wait for the links (the oldest group) only
#pragma unroll
    for (int D = 0; D < S - 1; ++D) {
        if (mask) issue(cur, D, D);
        __pipeline_commit();
    }
    __pipeline_wait_prior(S - 1);
    __syncthreads();  // every link of the tile is in shared memory
    if (!mask) return;
    int slot = 0;  // ring slot of the item being computed
    for (;;) {
        const int nxt = rest ? __ffs(rest) - 1 : -1;
        const int rhs = grp + cur * G;
        cplx<T> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};

#define LQ_SH_DIR(D)                                                                  \
    {                                                                                 \
        constexpr int MU = (D) >> 1;                                                  \
        constexpr bool FWD = ((D)&1) == 0;                                            \
        constexpr int SG = FWD ? SF : SB;                                             \
        {                                                                             \
            const int ahead = (D) + S - 1; /* item issued now: S - 1 ahead */         \
            int wslot = slot + S - 1;                                                 \
            if (wslot >= S) wslot -= S;                                               \
            if (ahead < 8) issue(cur, ahead, wslot);                                  \
            else if (nxt >= 0) issue(nxt, ahead - 8, wslot);                          \
        }                                                                             \
        __pipeline_commit();                                                          \
        __pipeline_wait_prior(S - 1);                                                 \
        const unsigned char* st = ring + slot * St::SPIN_BYTES;                       \
        cplx<T> sp[12], h[6], uh[6], u[9];                                            \
        T nrm;                                                                        \
        smem_spinor<P, R12, NT>(st, t, sp, nrm);                                      \
        project<MU, SG>(sp, h);                                                       \
        tile_link<P, R12>(links + (D)*LT::DIR, s, u);                                 \
        if (FWD ? sf[MU] : sb[MU]) {                                                  \
            _Pragma("unroll") for (int k = 0; k < 6; ++k) h[k] = cneg(h[k]);          \
        }                                                                             \
        su3_mul<!FWD>(u, h, uh);                                                      \
        reconstruct_add<MU, SG>(acc, uh);                                             \
        if (++slot == S) slot = 0;                                                    \
    }
        LQ_SH_DIR(0)
        LQ_SH_DIR(1)
        LQ_SH_DIR(2)
        LQ_SH_DIR(3)
        LQ_SH_DIR(4)
        LQ_SH_DIR(5)
        LQ_SH_DIR(6)
        LQ_SH_DIR(7)
#undef LQ_SH_DIR

        // epilogue of this right-hand side
        cplx<T> o[12];
        const T ch = (T)a.c_hop;
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = {ch * acc[k].re, ch * acc[k].im};
        if constexpr (EPI >= EPI_DIAG) {
            cplx<T> xs[12];
            T nx;
            load_spinor_raw<P, T>(a.x[p] + (size_t)rhs * a.x_rhs, g.Vh, i, xs, nx);
            const T cd = (T)a.c_diag * nx;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                o[k].re = fma(cd, xs[k].re, o[k].re);
                o[k].im = fma(cd, xs[k].im, o[k].im);
            }
        }
        if constexpr (EPI == EPI_DWF) {
            const int Ls = a.Ls, sl = rhs;
            const int s_up = DAG ? (sl + 1 == Ls ? 0 : sl + 1) : (sl == 0 ? Ls - 1 : sl - 1);
            const int s_dn = DAG ? (sl == 0 ? Ls - 1 : sl - 1) : (sl + 1 == Ls ? 0 : sl + 1);
            const bool wrap_up = DAG ? (sl + 1 == Ls) : (sl == 0);
            const bool wrap_dn = DAG ? (sl == 0) : (sl + 1 == Ls);
            const T c_up = wrap_up ? (T)(-a.c_shift * a.mf) : (T)a.c_shift;
            const T c_dn = wrap_dn ? (T)(-a.c_shift * a.mf) : (T)a.c_shift;
            cplx<T> su[6], sd[6];
            T nu, nd;
            // only P+ psi(s_up) (spins 0,1) and P- psi(s_dn) (spins 2,3) are needed
            load_half_spinor_raw<P, true>(a.x[p] + (size_t)s_up * a.x_rhs, g.Vh, i, su, nu);
            load_half_spinor_raw<P, false>(a.x[p] + (size_t)s_dn * a.x_rhs, g.Vh, i, sd, nd);
            const T cu = c_up * nu, cdn = c_dn * nd;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                o[k].re = fma(cu, su[k].re, o[k].re);
                o[k].im = fma(cu, su[k].im, o[k].im);
                o[6 + k].re = fma(cdn, sd[k].re, o[6 + k].re);
                o[6 + k].im = fma(cdn, sd[k].im, o[6 + k].im);
            }
        }
        if (active) store_spinor<P, T>(a.out[p] + (size_t)rhs * a.out_rhs, g.Vh, i, o);
        if constexpr (RED) {
            double v = 0;
            if (active) {
                T q = 0;
#pragma unroll
                for (int k = 0; k < 12; ++k) q += o[k].re * o[k].re + o[k].im * o[k].im;
                v = (double)q;
            }
            const int dwf = EPI == EPI_DWF;
            hop_norm_warp(v, a.red_partial, (int)shared_red_slot(a, dwf, rhs, pidx, tile * (NS / 32) + (s >> 5)));
            // the 128-site layout can have up to three more 32-site slots than the blocks'
            // warps fill: the last tile's warps write zeros there (the finalize sums every slot)
            const int tiles = (g.Vh + NS - 1) / NS;
            const int filled = tiles * (NS / 32), slots = ((g.Vh + kHopThreads - 1) / kHopThreads) * 4;
            if (tile == tiles - 1 && (t & 31) == 0)
                for (int c = filled + (s >> 5); c < slots; c += NS / 32)
                    a.red_partial[shared_red_slot(a, dwf, rhs, pidx, c)] = 0.0;
        }
        if (nxt < 0) break;
        cur = nxt;
        rest &= rest - 1;
    }
}

// Ring stages of the shared-link kernel: one spinor ahead.  Measured on
// 24^3 x 48 with 12 right-hand sides, two stages (525 us) beat three (533 us),
// whose larger shared-memory carve-out leaves less L1 for the epilogue's reads.
constexpr int kSharedStages = 2;

template <int P, bool R12, bool DAG, int EPI, bool RED>
cudaError_t launch_shared_one(const HopArgs& a, cudaStream_t st) {
    constexpr int G = kShGroups, NT = kShSites * G, S = kSharedStages;
    constexpr int smem = shared_smem_bytes<P, R12, NT, S>();
    auto kern = wilson_hop_shared_kernel<P, R12, DAG, EPI, G, S, RED>;
    static bool configured = false;  // attribute set once per process (per instantiation)
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int tiles = (a.g.Vh + kShSites - 1) / kShSites;
    return launch_pdl(kern, dim3(tiles * a.nparity), dim3(NT), smem, st, a);
}

// Does a launch go to the shared-link kernel?  Several right-hand sides (or
// slices) over whole parity blocks, at most 32 per group of threads.
inline bool hop_shared_applies(const HopArgs& a) {
    return a.nrhs >= 2 && a.nsite == 0 && a.site0 == 0 && a.nrhs <= 32 * kShGroups;
}

template <int P>
cudaError_t launch_hop_shared(const HopArgs& a, bool r12, bool dag, int epi, cudaStream_t st) {
    const bool red = a.red_partial != nullptr;
    if (red && epi == EPI_HOP) return cudaErrorInvalidValue;
#define LQ_S_EPI(R, D)                                                                       \
    switch (epi) {                                                                           \
    case EPI_HOP: return launch_shared_one<P, R, D, EPI_HOP, false>(a, st);                  \
    case EPI_DIAG: return red ? launch_shared_one<P, R, D, EPI_DIAG, true>(a, st)            \
                              : launch_shared_one<P, R, D, EPI_DIAG, false>(a, st);          \
    default: return red ? launch_shared_one<P, R, D, EPI_DWF, true>(a, st)                   \
                        : launch_shared_one<P, R, D, EPI_DWF, false>(a, st);                 \
    }
    if (r12) {
        if (dag) { LQ_S_EPI(true, true) } else { LQ_S_EPI(true, false) }
    } else {
        if (dag) { LQ_S_EPI(false, true) } else { LQ_S_EPI(false, false) }
    }
#undef LQ_S_EPI
}

}  // namespace lq
