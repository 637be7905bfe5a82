// hop_mma.cuh -- the multi-right-hand-side Wilson hop for FP16/BF16 storage
// with its SU(3) products on the tensor cores.
//
// With N right-hand sides sharing a link, the product of one site and one
// direction is a 3x3 complex matrix times 2 spins x N columns.  In real form
// it is Y^T = H^T B with
//   H^T: rows (spin, rhs), columns k = 2c + {re, im} of the input colour c;
//   B:   8 x 8, B[2c][2a] = Re U_ac, B[2c+1][2a] = -Im U_ac,
//        B[2c][2a+1] = Im U_ac, B[2c+1][2a+1] = Re U_ac (rows and columns 6, 7 zero);
// one mma.sync.m16n8k8 (16-bit inputs, FP32 accumulate) per site, direction
// and group of 8 right-hand sides: rows 0-7 are spin 0 of the group's right-hand
// sides, rows 8-15 spin 1.  In the fragment layout of that instruction, lane
// (g, q) = (lane / 4, lane % 4) holds A row g and g + 8 at columns 2q, 2q + 1,
// i.e. both spins of right-hand side g in colour q, and receives D at the same
// places.  So the spin projection (before) and the reconstruction with the
// site norm (after) stay lane-local; lanes with q = 3 carry the zero padding.
// The same lane holds B[2q][n], B[2q + 1][n] for n = g: one link word, with its
// halves swapped or a sign flipped.
//
// A block of 8 warps handles 32 sites x one group of 8 right-hand sides; each
// warp owns 4 of the sites and runs its own pipeline: its lanes copy the
// neighbour spinors, norms and links of one direction for its 4 sites x 8
// right-hand sides into the warp's ring of shared-memory stages with cp.async
// (lane l: site l % 4, right-hand side l / 4), three directions in flight, and
// only __syncwarp orders them -- no block barrier in the direction loop, so a
// warp waits on its own copies only, as in the CUDA-core hop.  The outputs
// leave through the warp's shared memory in the same order.  The block
// barrier at the end sums the fused norm over the block's 32 sites.
//
// Measured on 24^3 x 48 with 12 FP16 fields it takes 1.14 ms against 0.40 ms
// for the CUDA-core hop: the MMA replaces only the 72 FMAs of a site's SU(3)
// products, while the loads, projection and reconstruction, spread over three
// lanes per field, cost more instructions than the whole CUDA-core site.  It
// therefore runs only when a handle selects it (lq_set_hop_kernel).
#pragma once

#include <cuda_pipeline.h>

#include "lqcd_internal.cuh"
#include "lqcd_kernels.h"
#include "pdl.cuh"

namespace lq {

namespace mma {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kSitesPerWarp = 4;
constexpr int kSites = kSitesPerWarp * kWarps;  // sites per block
constexpr int kRhs = 8;                         // right-hand sides per block (one MMA row group)

// shared memory of one warp.  One stage: spinors [site][rhs][3 x 16 B] (site
// stride 400 B), norms [site][rhs], links [site][2 x 16 B + 4 B tail + 12 B pad].
constexpr int kSpnSite = kRhs * 48 + 16;
constexpr int kSpn = kSitesPerWarp * kSpnSite;
constexpr int kNrm = kSitesPerWarp * kRhs * 4;
constexpr int kLnk = kSitesPerWarp * 48;
constexpr int kStage = kSpn + kNrm + kLnk;
constexpr int kX = kSpn + kNrm;              // the diagonal input (EPI_DIAG)
constexpr int kNbr = kSitesPerWarp * 8 * 4;  // neighbour cb index per (site, direction)
constexpr int kSgn = kSitesPerWarp * 4;      // per site: bit D set = boundary phase -1 on direction D

__host__ __device__ constexpr int warp_bytes(int epi, int S) { return S * kStage + (epi == EPI_DIAG ? kX : 0) + kNbr + kSgn; }
constexpr int kRed = kWarps * kRhs * 4;  // per-warp, per-rhs |out|^2 (fused norm)
__host__ __device__ constexpr int smem_bytes(int epi, int S) { return kWarps * warp_bytes(epi, S) + kRed; }

template <int P>
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b) {
    if constexpr (P == LQ_F16)
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%7,%7,%7};"
                     : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
                     : "r"(a0), "r"(a1), "r"(b), "f"(0.f));
    else
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%7,%7,%7};"
                     : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
                     : "r"(a0), "r"(a1), "r"(b), "f"(0.f));
}

// the two projected spin components of colour q: (1 + S gamma_mu) psi = [h; S A^dag h],
// h = psi_up + S A_mu psi_dn, on packed halves as in project_h2
template <int P, int MU, int S>
__device__ __forceinline__ void project_colour(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3, uint32_t& h0,
                                               uint32_t& h1) {
    if constexpr (MU == 0) {
        h0 = h2_adds<P, -S>(p0, h2_mul_i(p3));
        h1 = h2_adds<P, -S>(p1, h2_mul_i(p2));
    } else if constexpr (MU == 1) {
        h0 = h2_adds<P, -S>(p0, p3);
        h1 = h2_adds<P, S>(p1, p2);
    } else if constexpr (MU == 2) {
        h0 = h2_adds<P, -S>(p0, h2_mul_i(p2));
        h1 = h2_adds<P, S>(p1, h2_mul_i(p3));
    } else {
        h0 = h2_adds<P, S>(p0, p2);
        h1 = h2_adds<P, S>(p1, p3);
    }
}

// acc (spins 0-3 of one colour, (re, im) pairs) += n [a; b; S A_mu^dag (a, b)], as reconstruct_fma
template <int MU, int S>
__device__ __forceinline__ void reconstruct_colour(float (&acc)[8], float ar, float ai, float br, float bi, float n) {
    const float sn = S > 0 ? n : -n;
    acc[0] = fmaf(n, ar, acc[0]);
    acc[1] = fmaf(n, ai, acc[1]);
    acc[2] = fmaf(n, br, acc[2]);
    acc[3] = fmaf(n, bi, acc[3]);
    if constexpr (MU == 0) {  // spin 2 += sn i b, spin 3 += sn i a
        acc[4] = fmaf(-sn, bi, acc[4]);
        acc[5] = fmaf(sn, br, acc[5]);
        acc[6] = fmaf(-sn, ai, acc[6]);
        acc[7] = fmaf(sn, ar, acc[7]);
    } else if constexpr (MU == 1) {  // spin 2 += sn b, spin 3 -= sn a
        acc[4] = fmaf(sn, br, acc[4]);
        acc[5] = fmaf(sn, bi, acc[5]);
        acc[6] = fmaf(-sn, ar, acc[6]);
        acc[7] = fmaf(-sn, ai, acc[7]);
    } else if constexpr (MU == 2) {  // spin 2 += sn i a, spin 3 -= sn i b
        acc[4] = fmaf(-sn, ai, acc[4]);
        acc[5] = fmaf(sn, ar, acc[5]);
        acc[6] = fmaf(sn, bi, acc[6]);
        acc[7] = fmaf(-sn, br, acc[7]);
    } else {  // spin 2 += sn a, spin 3 += sn b
        acc[4] = fmaf(sn, ar, acc[4]);
        acc[5] = fmaf(sn, ai, acc[5]);
        acc[6] = fmaf(sn, br, acc[6]);
        acc[7] = fmaf(sn, bi, acc[7]);
    }
}

}  // namespace mma

// grid.x = site tile x rhs group (groups fastest, so the groups of a tile share
// its links through L2), grid.y = output parity.  Requires a.nsite == 0.
template <int P, bool DAG, int EPI, bool RED, int MINB, int kStages>
__global__ void __launch_bounds__(mma::kThreads, MINB) wilson_hop_mma_kernel(const HopArgs a, int ngroups) {
    using namespace mma;
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned char* wsm = smem + warp * warp_bytes(EPI, kStages);
    unsigned char* xslot = wsm + kStages * kStage;
    int* nbr = reinterpret_cast<int*>(xslot + (EPI == EPI_DIAG ? kX : 0));
    unsigned* sgn = reinterpret_cast<unsigned*>(nbr + kSitesPerWarp * 8);
    float* red = reinterpret_cast<float*>(smem + kWarps * warp_bytes(EPI, kStages));

    const int tile = blockIdx.x / ngroups, grp = blockIdx.x - tile * ngroups;
    const int p = a.parity0 + blockIdx.y;
    const Geom& g = a.g;
    const int Vh = g.Vh;
    const int site0 = tile * kSites + warp * kSitesPerWarp;  // the warp's first site
    const int rhs0 = grp * kRhs;
    const int nr = min(kRhs, a.nrhs - rhs0);
    const int nsv = max(0, min(kSitesPerWarp, Vh - site0));  // valid sites of the warp

    pdl_enter();  // every global access of the block comes after this (programmatic dependent launch)
    // right-hand sides computed and stored (a set skip flag leaves one out; the domain wall's
    // slices share the flag of their 5-d system)
    const unsigned live =
        __ballot_sync(0xffffffffu, lane < nr && !(a.skip && a.skip[(EPI == EPI_DWF ? 0 : rhs0 + lane) * a.skip_stride])) &
        0xffu;
    if (live == 0) return;  // uniform over the block: every right-hand side of the group is finished
    if (lane < kSitesPerWarp) {
        unsigned bits = 0;
        int nf[4] = {0, 0, 0, 0}, nb[4] = {0, 0, 0, 0};
        if (lane < nsv) {
            const int i = site0 + lane;
            int x[4];
            cb_coords(g, i, p, x);
            const int xh = x[0] >> 1;
            int xf = x[0] + 1, xb = x[0] - 1;
            const bool sf = (xf == g.L[0]), sb = (xb < 0);
            if (sf) xf = 0;
            if (sb) xb = g.L[0] - 1;
            nf[0] = i - xh + (xf >> 1);
            nb[0] = i - xh + (xb >> 1);
            if (sf && g.bc[0] < 0) bits |= 1u;
            if (sb && g.bc[0] < 0) bits |= 2u;
            int step = g.Lh0;
#pragma unroll
            for (int mu = 1; mu < 4; ++mu) {
                const bool top = (x[mu] == g.L[mu] - 1), bot = (x[mu] == 0);
                nf[mu] = top ? i - (g.L[mu] - 1) * step : i + step;
                nb[mu] = bot ? i + (g.L[mu] - 1) * step : i - step;
                if (top && g.bc[mu] < 0) bits |= 1u << (2 * mu);
                if (bot && g.bc[mu] < 0) bits |= 2u << (2 * mu);
                step *= g.L[mu];
            }
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            nbr[lane * 8 + 2 * mu] = check_site(nf[mu], Vh);
            nbr[lane * 8 + 2 * mu + 1] = check_site(nb[mu], Vh);
        }
        sgn[lane] = bits;
    }
    __syncwarp();

    // staging roles: spinor chunks and norm of (site cs, rhs cr); lanes 0-11 the link chunks
    const int cs = lane & 3, cr = lane >> 2;
    const bool cp_spn = cs < nsv && ((live >> cr) & 1u);
    const char* __restrict__ in_r = a.in[p] + (size_t)(rhs0 + cr) * a.in_rhs;
    const char* __restrict__ Lp = a.links + (size_t)(p * 4) * a.link_block;
    const char* __restrict__ Lq = a.links + (size_t)((1 - p) * 4) * a.link_block;

    auto issue = [&](int D) {
        unsigned char* st = wsm + (D % kStages) * kStage;
        const int mu = D >> 1;
        const bool fwd = (D & 1) == 0;
        if (cp_spn) {
            const int ns = nbr[cs * 8 + D];
            unsigned char* dst = st + cs * kSpnSite + cr * 48;
#pragma unroll
            for (int k = 0; k < 3; ++k) __pipeline_memcpy_async(dst + 16 * k, in_r + ((size_t)k * Vh + ns) * 16, 16);
            __pipeline_memcpy_async(st + kSpn + (cs * kRhs + cr) * 4, in_r + (size_t)48 * Vh + (size_t)ns * 4, 4);
        }
        if (lane < 3 * kSitesPerWarp) {  // (site, part): parts 0, 1 the 16-byte chunks, 2 the 4-byte tail
            const int ls = lane & 3, lc = lane >> 2;
            if (ls < nsv) {
                const int li = fwd ? site0 + ls : nbr[ls * 8 + D];
                const char* lb = (fwd ? Lp : Lq) + (size_t)mu * a.link_block;
                unsigned char* dst = st + kSpn + kNrm + ls * 48;
                if (lc < 2) __pipeline_memcpy_async(dst + 16 * lc, lb + ((size_t)lc * Vh + li) * 16, 16);
                else __pipeline_memcpy_async(dst + 32, lb + (size_t)32 * Vh + (size_t)li * 4, 4);
            }
        }
    };

    issue(0);
    if constexpr (EPI == EPI_DIAG) {
        if (cp_spn) {
            const char* xr = a.x[p] + (size_t)(rhs0 + cr) * a.x_rhs;
            const int i = site0 + cs;
            unsigned char* dst = xslot + cs * kSpnSite + cr * 48;
#pragma unroll
            for (int k = 0; k < 3; ++k) __pipeline_memcpy_async(dst + 16 * k, xr + ((size_t)k * Vh + i) * 16, 16);
            __pipeline_memcpy_async(xslot + kSpn + (cs * kRhs + cr) * 4, xr + (size_t)48 * Vh + (size_t)i * 4, 4);
        }
    }
    __pipeline_commit();
#pragma unroll
    for (int D = 1; D < kStages - 1; ++D) {
        issue(D);
        __pipeline_commit();
    }

    const int gq = lane >> 2, q = lane & 3;  // right-hand side g (row), colour q (column pair)
    float acc[kSitesPerWarp][8];
#pragma unroll
    for (int m = 0; m < kSitesPerWarp; ++m)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[m][k] = 0.f;

    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    // iteration D: the stage of direction D - 1 is free once every lane is past its
    // compute (first __syncwarp); direction D's copies are complete for every lane
    // after its own wait (second __syncwarp)
#define LQ_MMA_DIR(D)                                                                                      \
    {                                                                                                      \
        constexpr int MU = (D) >> 1;                                                                       \
        constexpr bool FWD = ((D)&1) == 0;                                                                 \
        constexpr int SG = FWD ? SF : SB;                                                                  \
        __syncwarp();                                                                                      \
        if constexpr ((D) + kStages - 1 < 8) issue((D) + kStages - 1);                                    \
        __pipeline_commit();                                                                               \
        __pipeline_wait_prior(kStages - 1);                                                                \
        __syncwarp();                                                                                      \
        const unsigned char* st = wsm + ((D) % kStages) * kStage;                                          \
        _Pragma("unroll") for (int m = 0; m < kSitesPerWarp; ++m) {                                        \
            const uint32_t* L = reinterpret_cast<const uint32_t*>(st + kSpn + kNrm + m * 48);              \
            uint32_t b = 0;                                                                                \
            if (gq < 6 && q < 3) {                                                                         \
                const int aa = gq >> 1;                                                                    \
                if constexpr (FWD) {                                                                       \
                    const uint32_t w = L[aa * 3 + q];                                                      \
                    b = (gq & 1) ? __byte_perm(w, 0, 0x1032) : (w ^ 0x80000000u);                          \
                } else {                                                                                   \
                    const uint32_t w = L[q * 3 + aa];                                                      \
                    b = (gq & 1) ? (__byte_perm(w, 0, 0x1032) ^ 0x00008000u) : w;                          \
                }                                                                                          \
            }                                                                                              \
            uint32_t h0 = 0, h1 = 0;                                                                       \
            const uint32_t* sp = reinterpret_cast<const uint32_t*>(st + m * kSpnSite + gq * 48);           \
            if (q < 3) project_colour<P, MU, SG>(sp[q], sp[3 + q], sp[6 + q], sp[9 + q], h0, h1);          \
            float nrm = reinterpret_cast<const float*>(st + kSpn)[m * kRhs + gq];                          \
            if ((sgn[m] >> (D)) & 1u) nrm = -nrm;                                                          \
            float d[4];                                                                                    \
            mma16816<P>(d, h0, h1, b);                                                                     \
            reconstruct_colour<MU, SG>(acc[m], d[0], d[1], d[2], d[3], nrm);                               \
        }                                                                                                  \
    }
    LQ_MMA_DIR(0)
    LQ_MMA_DIR(1)
    LQ_MMA_DIR(2)
    LQ_MMA_DIR(3)
    LQ_MMA_DIR(4)
    LQ_MMA_DIR(5)
    LQ_MMA_DIR(6)
    LQ_MMA_DIR(7)
#undef LQ_MMA_DIR

    // epilogue: o = c_hop acc (+ c_diag x); the output goes through the warp's stage 0,
    // last read by direction 6, which every lane finished before the first __syncwarp
    // of direction 7
    __pipeline_wait_prior(0);
    std::integral_constant<int, P> tag;
    unsigned char* ost = wsm;
    const float ch = (float)a.c_hop;
    float rsum = 0.f;
#pragma unroll
    for (int m = 0; m < kSitesPerWarp; ++m) {
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = ch * acc[m][k];
        if constexpr (EPI == EPI_DIAG) {
            if (q < 3) {
                const uint32_t* xp = reinterpret_cast<const uint32_t*>(xslot + m * kSpnSite + gq * 48);
                const float cd = (float)a.c_diag * reinterpret_cast<const float*>(xslot + kSpn)[m * kRhs + gq];
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    const float2 v = h2f(xp[3 * sp + q], tag);
                    o[2 * sp] = fmaf(cd, v.x, o[2 * sp]);
                    o[2 * sp + 1] = fmaf(cd, v.y, o[2 * sp + 1]);
                }
            }
        }
        if constexpr (EPI == EPI_DWF) {
            // (5 - M5) psi(s) + c_up P+ psi(s_up) + c_dn P- psi(s_dn) at the lane's site, slice and
            // colour, read from the native blocks (mostly L2 hits: the slices of a tile run together)
            if (q < 3 && m < nsv && ((live >> gq) & 1u)) {
                const int i = site0 + m, Ls = a.Ls, sl = rhs0 + gq;
                const int s_up = DAG ? (sl + 1 == Ls ? 0 : sl + 1) : (sl == 0 ? Ls - 1 : sl - 1);
                const int s_dn = DAG ? (sl == 0 ? Ls - 1 : sl - 1) : (sl + 1 == Ls ? 0 : sl + 1);
                const bool wrap_up = DAG ? (sl + 1 == Ls) : (sl == 0);
                const bool wrap_dn = DAG ? (sl == 0) : (sl + 1 == Ls);
                const float c_up = wrap_up ? (float)(-a.c_shift * a.mf) : (float)a.c_shift;
                const float c_dn = wrap_dn ? (float)(-a.c_shift * a.mf) : (float)a.c_shift;
                auto word = [&](const char* blk, int c) {  // complex number c = 3 spin + colour of the site
                    return __ldg(reinterpret_cast<const uint32_t*>(blk + ((size_t)(c >> 2) * Vh + i) * 16) + (c & 3));
                };
                auto norm = [&](const char* blk) { return __ldg(reinterpret_cast<const float*>(blk + (size_t)48 * Vh) + i); };
                const char* xs = a.x[p] + (size_t)sl * a.x_rhs;
                const char* xu = a.x[p] + (size_t)s_up * a.x_rhs;
                const char* xd = a.x[p] + (size_t)s_dn * a.x_rhs;
                const float cd = (float)a.c_diag * norm(xs), cu = c_up * norm(xu), cdn = c_dn * norm(xd);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    const float2 v = h2f(word(xs, 3 * sp + q), tag);
                    o[2 * sp] = fmaf(cd, v.x, o[2 * sp]);
                    o[2 * sp + 1] = fmaf(cd, v.y, o[2 * sp + 1]);
                    // only P+ psi(s_up) (spins 0, 1) and P- psi(s_dn) (spins 2, 3)
                    const float2 w = h2f(word(sp < 2 ? xu : xd, 3 * sp + q), tag);
                    const float cw = sp < 2 ? cu : cdn;
                    o[2 * sp] = fmaf(cw, w.x, o[2 * sp]);
                    o[2 * sp + 1] = fmaf(cw, w.y, o[2 * sp + 1]);
                }
            }
        }
        float mx = 0.f, q2 = 0.f;
        if (q < 3) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                mx = fmaxf(mx, fabsf(o[k]));
                q2 += o[k] * o[k];
            }
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        if constexpr (RED) {
            q2 += __shfl_xor_sync(0xffffffffu, q2, 1);
            q2 += __shfl_xor_sync(0xffffffffu, q2, 2);
            if (m < nsv) rsum += q2;
        }
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint32_t* op = reinterpret_cast<uint32_t*>(ost + m * kSpnSite + gq * 48);
        if (q < 3) {
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) op[3 * sp + q] = f2h(o[2 * sp] * inv, o[2 * sp + 1] * inv, tag);
        }
        if (q == 0) reinterpret_cast<float*>(ost + kSpn)[m * kRhs + gq] = mx;
    }
    __syncwarp();
    if (cp_spn) {
        char* out_r = a.out[p] + (size_t)(rhs0 + cr) * a.out_rhs;
        const int i = site0 + cs;
        const uint4* src = reinterpret_cast<const uint4*>(ost + cs * kSpnSite + cr * 48);
#pragma unroll
        for (int k = 0; k < 3; ++k) reinterpret_cast<uint4*>(out_r + (size_t)k * Vh * 16)[i] = src[k];
        reinterpret_cast<float*>(out_r + (size_t)48 * Vh)[i] = reinterpret_cast<const float*>(ost + kSpn)[cs * kRhs + cr];
    }
    if constexpr (RED) {
        // one FP64 partial per (rhs, tile, parity) in the slots of the CUDA-core hop's warp
        // partials (hop_red_warps per rhs); tile 0 zeroes the slots no tile uses.  The domain
        // wall's one group holds the slices' slot sets one after another, so the same indexing
        // with the slice for the right-hand side fills it.
        if (q == 0) red[warp * kRhs + gq] = rsum;
        __syncthreads();
        const int nslots = ((Vh + kHopThreads - 1) / kHopThreads) * (kHopThreads / 32) * (int)gridDim.y;  // hop_red_warps
        const int ntiles = (Vh + kSites - 1) / kSites;
        if (t < kRhs && ((live >> t) & 1u)) {
            double v = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) v += (double)red[w * kRhs + t];
            double* base = a.red_partial + (size_t)(rhs0 + t) * nslots;
            base[tile * gridDim.y + blockIdx.y] = v;
            if (tile == 0 && blockIdx.y == 0)
                for (int k = ntiles * gridDim.y; k < nslots; ++k) base[k] = 0.0;
        }
    }
}

template <int P, bool DAG, int EPI, bool RED, int MINB, int S>
cudaError_t launch_mma_cfg(const HopArgs& a, cudaStream_t st) {
    constexpr int smem = mma::smem_bytes(EPI, S);
    auto kern = wilson_hop_mma_kernel<P, DAG, EPI, RED, MINB, S>;
    static bool configured = false;  // attribute set once per process (per instantiation)
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int ngroups = (a.nrhs + mma::kRhs - 1) / mma::kRhs;
    const int ntiles = (a.g.Vh + mma::kSites - 1) / mma::kSites;
    return launch_pdl(kern, dim3(ntiles * ngroups, a.nparity), dim3(mma::kThreads), smem, st, a, ngroups);
}

// 3 blocks of 8 warps per SM (80 registers) with 3 stages: measured on 24^3 x 48 x 8
// right-hand sides, 668 us against 787 us for 2 blocks with 3 or 4 stages
template <int P, bool DAG, int EPI, bool RED>
cudaError_t launch_mma_one(const HopArgs& a, cudaStream_t st) {
    return launch_mma_cfg<P, DAG, EPI, RED, 3, 3>(a, st);
}

// The tensor-core hop (selected with lq_set_hop_kernel) takes 18-real links, whole
// parity blocks and at least one full group of right-hand sides (or domain-wall
// slices, which share each link like right-hand sides).
inline bool hop_mma_applies(const HopArgs& a, bool r12, int epi) {
    (void)epi;
    return a.mma && !r12 && a.nsite == 0 && a.nrhs >= mma::kRhs;
}

template <int P>
cudaError_t launch_hop_mma(const HopArgs& a, bool dag, int epi, cudaStream_t st) {
    const bool red = a.red_partial != nullptr;
    if (red && epi == EPI_HOP) return cudaErrorInvalidValue;
    if (epi == EPI_DWF) {
        if (red) return dag ? launch_mma_one<P, true, EPI_DWF, true>(a, st) : launch_mma_one<P, false, EPI_DWF, true>(a, st);
        return dag ? launch_mma_one<P, true, EPI_DWF, false>(a, st) : launch_mma_one<P, false, EPI_DWF, false>(a, st);
    }
    if (epi == EPI_HOP) return dag ? launch_mma_one<P, true, EPI_HOP, false>(a, st) : launch_mma_one<P, false, EPI_HOP, false>(a, st);
    if (red) return dag ? launch_mma_one<P, true, EPI_DIAG, true>(a, st) : launch_mma_one<P, false, EPI_DIAG, true>(a, st);
    return dag ? launch_mma_one<P, true, EPI_DIAG, false>(a, st) : launch_mma_one<P, false, EPI_DIAG, false>(a, st);
}

}  // namespace lq
