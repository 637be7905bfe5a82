// hop_async.cuh -- the Wilson hop for FP32 / FP16 / BF16 storage with its
// neighbour gathers staged through shared memory by asynchronous copies.
//
// The single-right-hand-side hop is a bandwidth-bound gather: per output
// site it reads 8 neighbour spinors and 8 links.  Holding enough bytes in
// flight to cover HBM latency with plain loads costs registers (and so
// occupancy).  Here every thread streams its 8 (spinor, link) pairs through
// a private S-stage ring in shared memory with cp.async (16/8/4-byte
// copies that bypass the register file): the copies of directions D+1 ..
// D+S-1 are in flight while direction D is computed.  A thread reads back
// only the slots it filled itself, so no block-wide barrier is needed; the
// per-thread wait on its own copy groups (wait_prior) orders the data.
//
// Shared-memory layout of one stage: chunk-major [chunk][thread], 16-byte
// spinor chunks, then the site norms (FP16/BF16), then the link chunks, so a
// warp reading chunk k touches one contiguous 512-byte (or 256/128-byte) row.
#pragma once

#include <cuda_pipeline.h>

#include "lqcd_internal.cuh"
#include "lqcd_kernels.h"
#include "pdl.cuh"

namespace lq {

template <int P, bool R12>
struct AsyncLayout {
    static constexpr bool NORM = Prec<P>::has_norm;
    static constexpr int SP_CH = (P == LQ_F32) ? 6 : 3;  // 16-byte spinor chunks
    static constexpr int LK16 = LinkLayout<P, R12>::NFULL;  // 16-byte link chunks
    static constexpr int LKT = LinkLayout<P, R12>::TAIL;    // bytes of the link's tail chunk (0, 4, 8)
};

template <int P, bool R12, int NT>
struct AsyncStage {
    using L = AsyncLayout<P, R12>;
    static constexpr int SP_OFF = 0;
    static constexpr int NRM_OFF = SP_OFF + L::SP_CH * 16 * NT;
    static constexpr int LK_OFF = NRM_OFF + (L::NORM ? 4 * NT : 0);
    static constexpr int LKT_OFF = LK_OFF + L::LK16 * 16 * NT;
    static constexpr int BYTES = ((LKT_OFF + L::LKT * NT) + 15) / 16 * 16;
    static constexpr int SPIN_BYTES = ((L::SP_CH * 16 + (L::NORM ? 4 : 0)) * NT + 15) / 16 * 16;
    // half spinor (spins 0,1 or 2,3): FP32 3 x 16 B; FP16/BF16 16 + 8 B + norm
    static constexpr int HALF_BYTES = (((L::NORM ? 28 : 48)) * NT + 15) / 16 * 16;
};

// issue the copies of one spinor (all chunks + norm) into a spinor slot
template <int P, bool R12, int NT>
__device__ __forceinline__ void async_spinor(unsigned char* slot, const char* __restrict__ blk, int Vh, int site,
                                             int t) {
    using L = AsyncLayout<P, R12>;
    using St = AsyncStage<P, R12, NT>;
#pragma unroll
    for (int k = 0; k < L::SP_CH; ++k)
        __pipeline_memcpy_async(slot + St::SP_OFF + (k * NT + t) * 16, blk + ((size_t)k * Vh + site) * 16, 16);
    if constexpr (L::NORM)
        __pipeline_memcpy_async(slot + St::NRM_OFF + t * 4, blk + (size_t)48 * Vh + (size_t)site * 4, 4);
}

template <int P, bool R12, int NT>
__device__ __forceinline__ void async_link(unsigned char* stage, const char* __restrict__ blk, int Vh, int site,
                                           int t) {
    using L = AsyncLayout<P, R12>;
    using St = AsyncStage<P, R12, NT>;
#pragma unroll
    for (int c = 0; c < L::LK16; ++c)
        __pipeline_memcpy_async(stage + St::LK_OFF + (c * NT + t) * 16, blk + ((size_t)c * Vh + site) * 16, 16);
    if constexpr (L::LKT > 0)
        __pipeline_memcpy_async(stage + St::LKT_OFF + t * L::LKT,
                                blk + (size_t)L::LK16 * 16 * Vh + (size_t)site * L::LKT, L::LKT);
}

// issue the copies of the upper (spins 0,1) or lower (spins 2,3) half of a
// spinor into a half slot.  FP32: planes 0-2 or 3-5.  FP16/BF16 (3 planes of
// 4 complex): upper = plane 0 + the first 8 bytes of plane 1, lower = the last
// 8 bytes of plane 1 + plane 2.
template <int P, bool R12, int NT, bool UPPER>
__device__ __forceinline__ void async_half_spinor(unsigned char* slot, const char* __restrict__ blk, int Vh, int site,
                                                  int t) {
    using L = AsyncLayout<P, R12>;
    if constexpr (!L::NORM) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            __pipeline_memcpy_async(slot + (k * NT + t) * 16, blk + ((size_t)(UPPER ? k : 3 + k) * Vh + site) * 16, 16);
    } else {
        __pipeline_memcpy_async(slot + t * 16, blk + ((size_t)(UPPER ? 0 : 2) * Vh + site) * 16, 16);
        __pipeline_memcpy_async(slot + 16 * NT + t * 8, blk + ((size_t)Vh + site) * 16 + (UPPER ? 0 : 8), 8);
        __pipeline_memcpy_async(slot + 24 * NT + t * 4, blk + (size_t)48 * Vh + (size_t)site * 4, 4);
    }
}

// read a staged half spinor back: 6 complex in spin-colour order of its half
template <int P, bool R12, int NT, bool UPPER>
__device__ __forceinline__ void smem_half_spinor(const unsigned char* slot, int t, cplx<float> (&s)[6], float& nrm) {
    using L = AsyncLayout<P, R12>;
    if constexpr (!L::NORM) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = *reinterpret_cast<const float4*>(slot + (k * NT + t) * 16);
            s[2 * k] = {v.x, v.y};
            s[2 * k + 1] = {v.z, v.w};
        }
        nrm = 1.f;
    } else {
        std::integral_constant<int, P> tag;
        const uint4 v = *reinterpret_cast<const uint4*>(slot + t * 16);
        const uint2 w = *reinterpret_cast<const uint2*>(slot + 16 * NT + t * 8);
        const float2 q0 = h2f(v.x, tag), q1 = h2f(v.y, tag), q2 = h2f(v.z, tag), q3 = h2f(v.w, tag);
        const float2 r0 = h2f(w.x, tag), r1 = h2f(w.y, tag);
        const int a = UPPER ? 0 : 2, b = UPPER ? 4 : 0;  // where the 16-byte and the 8-byte parts go
        s[a + 0] = {q0.x, q0.y};
        s[a + 1] = {q1.x, q1.y};
        s[a + 2] = {q2.x, q2.y};
        s[a + 3] = {q3.x, q3.y};
        s[b + 0] = {r0.x, r0.y};
        s[b + 1] = {r1.x, r1.y};
        nrm = *reinterpret_cast<const float*>(slot + 24 * NT + t * 4);
    }
}

// the upper (spins 0,1) or lower (spins 2,3) half of a spinor straight from its
// native block, in the order of smem_half_spinor (unscaled values + norm)
template <int P, bool UPPER>
__device__ __forceinline__ void load_half_spinor_raw(const char* __restrict__ blk, int Vh, int i, cplx<float> (&s)[6],
                                                     float& nrm) {
    if constexpr (P == LQ_F32) {
        const float4* q = reinterpret_cast<const float4*>(blk);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = __ldg(q + (size_t)(UPPER ? k : 3 + k) * Vh + i);
            s[2 * k] = {v.x, v.y};
            s[2 * k + 1] = {v.z, v.w};
        }
        nrm = 1.f;
    } else {
        std::integral_constant<int, P> tag;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(blk) + (size_t)(UPPER ? 0 : 2) * Vh + i);
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(blk + ((size_t)Vh + i) * 16) + (UPPER ? 0 : 1));
        const float2 q0 = h2f(v.x, tag), q1 = h2f(v.y, tag), q2 = h2f(v.z, tag), q3 = h2f(v.w, tag);
        const float2 r0 = h2f(w.x, tag), r1 = h2f(w.y, tag);
        const int a = UPPER ? 0 : 2, b = UPPER ? 4 : 0;  // where the 16-byte and the 8-byte parts go
        s[a + 0] = {q0.x, q0.y};
        s[a + 1] = {q1.x, q1.y};
        s[a + 2] = {q2.x, q2.y};
        s[a + 3] = {q3.x, q3.y};
        s[b + 0] = {r0.x, r0.y};
        s[b + 1] = {r1.x, r1.y};
        nrm = __ldg(reinterpret_cast<const float*>(blk + (size_t)48 * Vh) + i);
    }
}

// read one staged spinor back (unscaled values + norm)
template <int P, bool R12, int NT>
__device__ __forceinline__ void smem_spinor(const unsigned char* slot, int t, cplx<float> (&s)[12], float& nrm) {
    using L = AsyncLayout<P, R12>;
    using St = AsyncStage<P, R12, NT>;
    if constexpr (P == LQ_F32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = *reinterpret_cast<const float4*>(slot + St::SP_OFF + (k * NT + t) * 16);
            s[2 * k] = {v.x, v.y};
            s[2 * k + 1] = {v.z, v.w};
        }
        nrm = 1.f;
    } else {
        std::integral_constant<int, P> tag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 v = *reinterpret_cast<const uint4*>(slot + St::SP_OFF + (k * NT + t) * 16);
            float2 a = h2f(v.x, tag), b = h2f(v.y, tag), c = h2f(v.z, tag), d = h2f(v.w, tag);
            s[4 * k + 0] = {a.x, a.y};
            s[4 * k + 1] = {b.x, b.y};
            s[4 * k + 2] = {c.x, c.y};
            s[4 * k + 3] = {d.x, d.y};
        }
        nrm = *reinterpret_cast<const float*>(slot + St::NRM_OFF + t * 4);
    }
    (void)sizeof(L);
}

template <int P, bool R12, int NT>
__device__ __forceinline__ void smem_link(const unsigned char* stage, int t, cplx<float> (&u)[9]) {
    using L = AsyncLayout<P, R12>;
    using St = AsyncStage<P, R12, NT>;
    RawLink<P, R12> r;
#pragma unroll
    for (int c = 0; c < L::LK16; ++c) {
        const uint4 v = *reinterpret_cast<const uint4*>(stage + St::LK_OFF + (c * NT + t) * 16);
        r.w[4 * c] = v.x;
        r.w[4 * c + 1] = v.y;
        r.w[4 * c + 2] = v.z;
        r.w[4 * c + 3] = v.w;
    }
    if constexpr (L::LKT == 8) {
        const uint2 v = *reinterpret_cast<const uint2*>(stage + St::LKT_OFF + t * 8);
        r.w[4 * L::LK16] = v.x;
        r.w[4 * L::LK16 + 1] = v.y;
    } else if constexpr (L::LKT == 4) {
        r.w[4 * L::LK16] = *reinterpret_cast<const uint32_t*>(stage + St::LKT_OFF + t * 4);
    }
    raw_unpack<P, R12, float>(r, u);
}

// staged FP16/BF16 spinor as 12 packed complex words + norm
template <int P, int NT>
__device__ __forceinline__ void smem_words_spinor(const unsigned char* slot, int t, uint32_t (&w)[12], float& nrm) {
    using St = AsyncStage<P, false, NT>;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 v = *reinterpret_cast<const uint4*>(slot + St::SP_OFF + (k * NT + t) * 16);
        w[4 * k] = v.x;
        w[4 * k + 1] = v.y;
        w[4 * k + 2] = v.z;
        w[4 * k + 3] = v.w;
    }
    nrm = *reinterpret_cast<const float*>(slot + St::NRM_OFF + t * 4);
}

// staged FP16/BF16 18-real link as 9 packed complex words
template <int P, int NT>
__device__ __forceinline__ void smem_words_link(const unsigned char* stage, int t, uint32_t (&w)[9]) {
    using St = AsyncStage<P, false, NT>;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint4 v = *reinterpret_cast<const uint4*>(stage + St::LK_OFF + (c * NT + t) * 16);
        w[4 * c] = v.x;
        w[4 * c + 1] = v.y;
        w[4 * c + 2] = v.z;
        w[4 * c + 3] = v.w;
    }
    w[8] = *reinterpret_cast<const uint32_t*>(stage + St::LKT_OFF + t * 4);
}

// Whether the diagonal input rides with direction 0 through shared memory.  The
// FP16/BF16 hop reads it from global memory in the epilogue instead: a staged
// copy costs it a block of residency per SM (5 instead of 6), and on 32^4 its
// Schur step is 3% faster without (36.6 -> 35.4 us per hop); FP32 (2 stages,
// not limited by shared memory) is faster staged, most on L2-resident lattices
// (16^3 x 32: 8.7 against 9.6 us).  The domain-wall epilogue stages its three
// spinor inputs.
template <int P, int EPI>
__host__ __device__ constexpr bool stage_x() {
    return EPI == EPI_DIAG && !Prec<P>::has_norm;
}

template <int P, bool R12, int NT, int EPI>
constexpr int async_smem_bytes(int S) {
    using St = AsyncStage<P, R12, NT>;
    return S * St::BYTES + (stage_x<P, EPI>() ? St::SPIN_BYTES : 0);
}

// launch configuration per storage precision: threads per block, stages.
// Fewer stages leave room for more resident blocks; on 32^4 (one rhs) and
// 24^3x48 (12 rhs) FP32 is fastest with 2 stages and FP16/BF16 with 3
// (FP32 3 -> 2: 12 rhs 652 -> 626 us; FP16 4 -> 3: 437 -> 414 us, 37.5 -> 37.0 us).
template <int P>
struct AsyncCfg {
    static constexpr int NT = kHopThreads;
    static constexpr int S = (P == LQ_F32) ? 2 : 3;
};

// stages of every variant.  The domain-wall epilogue reads its three extra
// spinor inputs (psi(s) and the halves of psi(s -+ 1)) from global memory, where
// they are mostly L2 hits (the slices of a site tile run together), instead of
// staging them: on 16^4 x 16 that took FP32 from 96 to 87 us (5 blocks per SM
// instead of 3); FP16 stayed at 59 us with 2 or 3 stages.
template <int P, int EPI>
constexpr int async_stages() {
    return AsyncCfg<P>::S;
}

// One output site (checkerboard index i < Vh, right-hand side rhs, parity p):
// the staged 8-direction gather and the epilogue, result in o (not stored).
template <int P, bool R12, bool DAG, int EPI, int NT, int S>
__device__ __forceinline__ void hop_async_site(const HopArgs& a, int i, int rhs, int p, unsigned char* smem, int t,
                                               cplx<float> (&o)[12]) {
    using T = float;
    using St = AsyncStage<P, R12, NT>;
    const Geom& g = a.g;
    const char* __restrict__ in = a.in[p] + (size_t)rhs * a.in_rhs;
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
    unsigned char* extra = smem + S * St::BYTES;  // diagonal / 5th-dimension spinors

    auto issue = [&](int D) {
        unsigned char* stage = smem + (D % S) * St::BYTES;
        const int mu = D >> 1;
        const bool fwd = (D & 1) == 0;
        async_spinor<P, R12, NT>(stage, in, g.Vh, fwd ? nf[mu] : nb[mu], t);
        async_link<P, R12, NT>(stage, (fwd ? Lp : Lq) + (size_t)mu * a.link_block, g.Vh, fwd ? i : nb[mu], t);
    };

    // prologue: the diagonal / 5th-dimension inputs ride with direction 0
    issue(0);
    int s_up = 0, s_dn = 0;
    T c_up = 0, c_dn = 0;
    if constexpr (stage_x<P, EPI>()) {
        async_spinor<P, R12, NT>(extra, a.x[p] + (size_t)rhs * a.x_rhs, g.Vh, i, t);
    }
    if constexpr (EPI == EPI_DWF) {
        const int Ls = a.Ls;
        const int sl = rhs;
        s_up = DAG ? (sl + 1 == Ls ? 0 : sl + 1) : (sl == 0 ? Ls - 1 : sl - 1);
        s_dn = DAG ? (sl == 0 ? Ls - 1 : sl - 1) : (sl + 1 == Ls ? 0 : sl + 1);
        const bool wrap_up = DAG ? (sl + 1 == Ls) : (sl == 0);
        const bool wrap_dn = DAG ? (sl == 0) : (sl + 1 == Ls);
        c_up = wrap_up ? (T)(-a.c_shift * a.mf) : (T)a.c_shift;
        c_dn = wrap_dn ? (T)(-a.c_shift * a.mf) : (T)a.c_shift;
    }
    __pipeline_commit();
#pragma unroll
    for (int D = 1; D < S - 1; ++D) {
        issue(D);
        __pipeline_commit();
    }

    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    constexpr bool NORM = Prec<P>::has_norm;
    // FP16/BF16 with 18-real links: packed projection and mixed-precision FMAs
    constexpr bool PACKED = NORM && !R12;
    cplx<T> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};

#define LQ_ASYNC_DIR(D)                                                               \
    {                                                                                 \
        constexpr int MU = (D) >> 1;                                                  \
        constexpr bool FWD = ((D)&1) == 0;                                            \
        constexpr int SG = FWD ? SF : SB;                                             \
        if constexpr ((D) + S - 1 < 8) issue((D) + S - 1);                            \
        __pipeline_commit();                                                          \
        __pipeline_wait_prior(S - 1);                                                 \
        const unsigned char* stage = smem + ((D) % S) * St::BYTES;                    \
        cplx<T> s[12], h[6], uh[6], u[9];                                             \
        T nrm;                                                                        \
        const bool sgn = FWD ? sf[MU] : sb[MU];                                       \
        if constexpr (PACKED) {                                                       \
            uint32_t sw[12], hw[6], uw[9];                                            \
            smem_words_spinor<P, NT>(stage, t, sw, nrm);                              \
            project_h2<P, MU, SG>(sw, hw);                                            \
            smem_words_link<P, NT>(stage, t, uw);                                     \
            su3_mul_h2<P, !FWD>(uw, hw, uh);                                          \
            reconstruct_fma<MU, SG>(acc, uh, sgn ? -nrm : nrm);                       \
        } else if constexpr (NORM) {                                                  \
            smem_spinor<P, R12, NT>(stage, t, s, nrm);                                \
            project<MU, SG>(s, h);                                                    \
            smem_link<P, R12, NT>(stage, t, u);                                       \
            su3_mul<!FWD>(u, h, uh);                                                  \
            reconstruct_fma<MU, SG>(acc, uh, sgn ? -nrm : nrm);                       \
        } else {                                                                      \
            smem_spinor<P, R12, NT>(stage, t, s, nrm);                                \
            project<MU, SG>(s, h);                                                    \
            smem_link<P, R12, NT>(stage, t, u);                                       \
            if (sgn) {                                                                \
                _Pragma("unroll") for (int k = 0; k < 6; ++k) h[k] = cneg(h[k]);      \
            }                                                                         \
            su3_mul<!FWD>(u, h, uh);                                                  \
            reconstruct_add<MU, SG>(acc, uh);                                         \
        }                                                                             \
    }
    LQ_ASYNC_DIR(0)
    LQ_ASYNC_DIR(1)
    LQ_ASYNC_DIR(2)
    LQ_ASYNC_DIR(3)
    LQ_ASYNC_DIR(4)
    LQ_ASYNC_DIR(5)
    LQ_ASYNC_DIR(6)
    LQ_ASYNC_DIR(7)
#undef LQ_ASYNC_DIR

    const T ch = (T)a.c_hop;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = {ch * acc[k].re, ch * acc[k].im};
    if constexpr (EPI >= EPI_DIAG) {
        cplx<T> xs[12];
        T nx;
        if constexpr (stage_x<P, EPI>()) smem_spinor<P, R12, NT>(extra, t, xs, nx);
        else load_spinor_raw<P, T>(a.x[p] + (size_t)rhs * a.x_rhs, g.Vh, i, xs, nx);
        const T cd = (T)a.c_diag * nx;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            o[k].re = fma(cd, xs[k].re, o[k].re);
            o[k].im = fma(cd, xs[k].im, o[k].im);
        }
    }
    if constexpr (EPI == EPI_DWF) {
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
}

template <int P, bool R12, bool DAG, int EPI, int NT, int S, bool RED>
__global__ void __launch_bounds__(NT) wilson_hop_async_kernel(const HopArgs a) {
    using T = float;
    extern __shared__ __align__(16) unsigned char smem[];
    // grid.x = (rhs, output parity, site tile), rhs fastest: the right-hand sides, or
    // 5th-dimension slices, of one site tile run together and share each link through
    // L2/L1, and so do the two parities of a tile (one parity's outputs read the other's
    // block as neighbours, its own as the diagonal / 5th-dimension input).  With the
    // parities in separate passes a full-lattice launch read its input and links twice.
    const int t = threadIdx.x;
    const int rhs = blockIdx.x % a.nrhs;
    const int pt = blockIdx.x / a.nrhs;  // parity x tile index
    const Geom& g = a.g;
    const int end = a.nsite ? a.site0 + a.nsite : g.Vh;
    const int i0 = a.site0 + (pt / a.nparity) * NT + t;
    const bool active = i0 < end;
    // without the fused norm there is no block barrier: a thread past the end leaves;
    // with it, such a thread recomputes the last site and stores nothing
    if constexpr (!RED) {
        if (!active) return;
    }
    const int i = active ? i0 : end - 1;
    const int p = a.parity0 + pt % a.nparity;
    pdl_enter();  // every global access of the block comes after this (programmatic dependent launch)
    if (a.skip && a.skip[(EPI == EPI_DWF ? 0 : rhs) * a.skip_stride]) return;  // uniform per block
    cplx<T> o[12];
    hop_async_site<P, R12, DAG, EPI, NT, S>(a, i, rhs, p, smem, t, o);
    if (active) store_spinor<P, T>(a.out[p] + (size_t)rhs * a.out_rhs, g.Vh, i, o);
    if constexpr (RED) {
        double v = 0;
        if (active) {
            T q = 0;
#pragma unroll
            for (int k = 0; k < 12; ++k) q += o[k].re * o[k].re + o[k].im * o[k].im;
            v = (double)q;
        }
        // warp partials, group-major: [group][warp of the group's blocks]
        const int wpb = blockDim.x >> 5;
        const int grp = EPI == EPI_DWF ? 0 : rhs;
        const int nblk = EPI == EPI_DWF ? gridDim.x : gridDim.x / a.nrhs;
        const int bidx = EPI == EPI_DWF ? blockIdx.x : pt;
        hop_norm_warp(v, a.red_partial + (size_t)grp * nblk * wpb, bidx * wpb + (threadIdx.x >> 5));
    }
}

template <int P, bool R12, bool DAG, int EPI, bool RED>
cudaError_t launch_async_one(const HopArgs& a, cudaStream_t st) {
    constexpr int NT = AsyncCfg<P>::NT, S = async_stages<P, EPI>();
    constexpr int smem = async_smem_bytes<P, R12, NT, EPI>(S);
    auto kern = wilson_hop_async_kernel<P, R12, DAG, EPI, NT, S, RED>;
    static bool configured = false;  // attribute set once per process (per instantiation)
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int nsite = a.nsite ? a.nsite : a.g.Vh;
    return launch_pdl(kern, dim3(((nsite + NT - 1) / NT) * a.nrhs * a.nparity), dim3(NT), smem, st, a);
}

// ---------------------------------------------------------------------------
// Persistent hop over a batch of lattices of different sizes: one launch of
// `grid` blocks walks the flattened work list of every lattice's
// (site tile, right-hand side, parity) items, tile = batch_mult x NT sites
// (each lattice its own, chosen by the autotuner), item k of lattice l at
// lat_off[l] + k.  The per-lattice launch descriptors (pointers, geometry,
// links, skip flags, tile size) live in device memory.
template <int P, bool R12, bool DAG, int EPI, int NT, int S>
__global__ void __launch_bounds__(NT) wilson_hop_batch_kernel(const HopArgs* __restrict__ args,
                                                              const int* __restrict__ lat_off, int nlat) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x;
    const int total = lat_off[nlat];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int l = 0;
        while (l + 1 < nlat && item >= lat_off[l + 1]) ++l;
        const HopArgs& a = args[l];
        int local = item - lat_off[l];
        const int pidx = local % a.nparity;
        local /= a.nparity;
        const int rhs = local % a.nrhs;
        const int tile = local / a.nrhs;
        if (a.skip && a.skip[rhs * a.skip_stride]) continue;
        const int p = a.parity0 + pidx;
        const int mult = a.batch_mult;
        for (int m = 0; m < mult; ++m) {
            const int i = (tile * mult + m) * NT + t;
            if (i < a.g.Vh) {
                cplx<float> o[12];
                hop_async_site<P, R12, DAG, EPI, NT, S>(a, i, rhs, p, smem, t, o);
                store_spinor<P, float>(a.out[p] + (size_t)rhs * a.out_rhs, a.g.Vh, i, o);
            }
        }
    }
}

template <int P, bool R12, bool DAG, int EPI>
cudaError_t launch_batch_one(const HopArgs* args, const int* lat_off, int nlat, int grid, cudaStream_t st,
                             int* max_blocks_per_sm) {
    constexpr int NT = AsyncCfg<P>::NT, S = AsyncCfg<P>::S;
    constexpr int smem = async_smem_bytes<P, R12, NT, EPI>(S);
    auto kern = wilson_hop_batch_kernel<P, R12, DAG, EPI, NT, S>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (max_blocks_per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, kern, NT, smem);
    kern<<<grid, NT, smem, st>>>(args, lat_off, nlat);
    return cudaGetLastError();
}

// Batched hop launch (grid = 0: report the occupancy in *max_blocks_per_sm instead).
template <int P>
cudaError_t launch_hop_batch_prec(const HopArgs* args, const int* lat_off, int nlat, bool r12, bool dag, int epi,
                                  int grid, cudaStream_t st, int* max_blocks_per_sm) {
    if (epi == EPI_DWF) return cudaErrorInvalidValue;
#define LQ_B_EPI(R, D)                                                                                       \
    return epi == EPI_HOP ? launch_batch_one<P, R, D, EPI_HOP>(args, lat_off, nlat, grid, st, max_blocks_per_sm) \
                          : launch_batch_one<P, R, D, EPI_DIAG>(args, lat_off, nlat, grid, st, max_blocks_per_sm);
    if (r12) {
        if (dag) { LQ_B_EPI(true, true) } else { LQ_B_EPI(true, false) }
    } else {
        if (dag) { LQ_B_EPI(false, true) } else { LQ_B_EPI(false, false) }
    }
#undef LQ_B_EPI
}

template <int P>
cudaError_t launch_hop_async(const HopArgs& a, bool r12, bool dag, int epi, cudaStream_t st) {
    const bool red = a.red_partial != nullptr;
    if (red && epi == EPI_HOP) return cudaErrorInvalidValue;
#define LQ_A_EPI(R, D)                                                                       \
    switch (epi) {                                                                           \
    case EPI_HOP: return launch_async_one<P, R, D, EPI_HOP, false>(a, st);                   \
    case EPI_DIAG: return red ? launch_async_one<P, R, D, EPI_DIAG, true>(a, st)             \
                              : launch_async_one<P, R, D, EPI_DIAG, false>(a, st);           \
    default: return red ? launch_async_one<P, R, D, EPI_DWF, true>(a, st)                    \
                        : launch_async_one<P, R, D, EPI_DWF, false>(a, st);                  \
    }
    if (r12) {
        if (dag) { LQ_A_EPI(true, true) } else { LQ_A_EPI(true, false) }
    } else {
        if (dag) { LQ_A_EPI(false, true) } else { LQ_A_EPI(false, false) }
    }
#undef LQ_A_EPI
}

}  // namespace lq
