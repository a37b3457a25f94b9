// Per-tile arithmetic of the ray -> voxel message kernels (Eqs. "pos"/"neg").
//
// Notation for one ray with voxels i = 1..N in order of range:
//   m1_i = mu_{o_i -> psi}(1) = sigmoid(L_i), m0_i = 1 - m1_i, L_i the cavity log-odds
//   nu_i  sensor likelihood of a surface in voxel i; nu_bg the all-empty term
//   P_i = prod_{k<i} m0_k            (visibility up to voxel i)
//   A_i = sum_{j<i} m1_j nu_j P_j    (evidence of a surface before voxel i;
//                                     the summand is Eq. "depth_message")
//   B_i = sum_{j>i} m1_j nu_j prod_{i<k<j} m0_k + nu_bg prod_{k>i} m0_k
// Eqs. "pos"/"neg" then read pos_i = A_i + P_i nu_i and
// neg_i = A_i + P_i B_i (the 1/mu(o_i=0) of Eq. "neg" cancels the m0_i inside
// P_j for j > i), and the message is lambda_i = log(pos_i / neg_i).
//
// A and P are a forward linear recurrence, (A, P) <- (A + P m1 nu, P m0);
// B is a backward one, B <- m1 nu + m0 B, started at nu_bg.  Every quantity
// stays bounded: P is a probability, A <= max nu, B lies between the smallest
// and largest nu on the ray.  So both scans run in plain FP32 without
// log-domain rescaling; the transcendentals per edge are one exp and one
// reciprocal (for m1, m0) and one reciprocal and one log (for lambda).
//
// A tile is a run of whole rays; each of the CTA's 256 threads holds KT
// consecutive edges, scans them sequentially, and the CTA combines the
// thread aggregates with warp shuffles (segmented by ray starts and ends).
#pragma once

#include "mrf_internal.cuh"

namespace mrf {
namespace tile {

struct Fwd {   // map (A, P) -> (A + x P, y P), or a reset to the ray start if h
    float x, y;
    int h;
};
struct Bwd {   // map B -> u + v B, or constant u if h (v = 0)
    float u, v;
    int h;
};

__device__ __forceinline__ Fwd fwd_op(const Fwd &a, const Fwd &b) {  // a precedes b
    if (b.h) return b;
    return {fmaf(a.y, b.x, a.x), a.y * b.y, a.h};
}
__device__ __forceinline__ Bwd bwd_op(const Bwd &lo, const Bwd &hi) {  // hi is applied first
    if (lo.h) return lo;
    return {fmaf(lo.v, hi.u, lo.u), lo.v * hi.v, hi.h};
}
__device__ __forceinline__ Fwd shfl_up(const Fwd &a, int o) {
    return {__shfl_up_sync(0xffffffffu, a.x, o), __shfl_up_sync(0xffffffffu, a.y, o),
            __shfl_up_sync(0xffffffffu, a.h, o)};
}
__device__ __forceinline__ Bwd shfl_down(const Bwd &a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.u, o), __shfl_down_sync(0xffffffffu, a.v, o),
            __shfl_down_sync(0xffffffffu, a.h, o)};
}

// Exclusive forward scan over the CTA's threads (thread 0 gets the identity).
// Warps scan with shuffles; warp 0 then scans the 8 warp totals.
__device__ __forceinline__ Fwd block_fwd_exclusive(Fwd v, Fwd *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Fwd inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Fwd y = shfl_up(inc, o);
        if (lane >= o) inc = fwd_op(y, inc);
    }
    Fwd ex = shfl_up(inc, 1);
    if (lane == 0) ex = {0.f, 1.f, 0};
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        constexpr int NWARP = kThreads / 32;
        Fwd t = lane < NWARP ? s_w[lane] : Fwd{0.f, 1.f, 0};
#pragma unroll
        for (int o = 1; o < NWARP; o <<= 1) {
            const Fwd y = shfl_up(t, o);
            if (lane >= o) t = fwd_op(y, t);
        }
        Fwd e = shfl_up(t, 1);
        if (lane == 0) e = {0.f, 1.f, 0};
        if (lane < NWARP) s_w[NWARP + lane] = e;
    }
    __syncthreads();
    return fwd_op(s_w[kThreads / 32 + warp], ex);
}

// Exclusive backward (suffix) scan: the composition of every later thread's map.
__device__ __forceinline__ Bwd block_bwd_exclusive(Bwd v, Bwd *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Bwd inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Bwd y = shfl_down(inc, o);
        if (lane + o < 32) inc = bwd_op(inc, y);
    }
    Bwd ex = shfl_down(inc, 1);
    if (lane == 31) ex = {0.f, 1.f, 0};
    if (lane == 0) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        constexpr int NWARP = kThreads / 32;
        Bwd t = lane < NWARP ? s_w[lane] : Bwd{0.f, 1.f, 0};
#pragma unroll
        for (int o = 1; o < NWARP; o <<= 1) {
            const Bwd y = shfl_down(t, o);
            if (lane + o < NWARP) t = bwd_op(t, y);
        }
        Bwd e = shfl_down(t, 1);
        if (lane == NWARP - 1) e = {0.f, 1.f, 0};
        if (lane < NWARP) s_w[NWARP + lane] = e;
    }
    __syncthreads();
    return bwd_op(ex, s_w[kThreads / 32 + warp]);
}

// One step of the visibility product, P <- P m0, and of the backward state,
// B <- m1 nu + m0 B = B + m1 (nu - B).  A free-space voxel has m0 = 1 - m1 with
// m1 tiny, and m0 stored in FP32 keeps only a few digits of m1; so when m1 < 1/2
// the steps are taken through m1 with one rounding (fmaf), and through m0
// otherwise (where m0 is the small, precise one).
__device__ __forceinline__ float step_P(float P, float m0, float m1) {
    return m1 < 0.5f ? fmaf(-P, m1, P) : P * m0;
}
__device__ __forceinline__ float step_B(float B, float m0, float m1, float c, float nu) {
    return m1 < 0.5f ? fmaf(m1, nu - B, B) : fmaf(m0, B, c);
}

// 1/x to about 1 ulp for x in [1e-30, 1e30]: the hardware reciprocal estimate
// refined by one Newton step (outside that range, where the estimate flushes,
// the correctly rounded reciprocal).
__device__ __forceinline__ float recip(float x) {
    if (!(x > 1e-30f && x < 1e30f)) return __frcp_rn(x);
    const float r = __fdividef(1.f, x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// The same for x in [1, 2], where the estimate never flushes.
__device__ __forceinline__ float recip_1_2(float x) {
    const float r = __fdividef(1.f, x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// lambda = log(pos / neg) from pos = A + P nu and neg = A + P B.  With
// q = (pos - neg) / neg = P (nu - B) / neg, log(1 + q) is formed as
// log(u) + (q - (u - 1)) / u with u = fl(1 + q), which keeps full relative
// precision for the many near-zero messages; where q <= -1/2 (pos well below
// neg) 1 + q would lose bits and u = pos / neg, a ratio of two non-negative
// sums, is used directly.  neg = 0 (possible only when nu_bg = 0) gives +64, or
// 0 when pos is 0 as well.
__device__ __forceinline__ float message(float A, float P, float nu, float B) {
    const float num = fmaf(P, nu, A);
    const float den = fmaf(P, B, A);
    if (!(den > 0.f)) return num > 0.f ? kLamClamp : 0.f;
    const float rden = recip(den);
    const float q = P * (nu - B) * rden;
    float u, corr = 0.f;
    if (q > -0.5f) {
        u = 1.f + q;
        if (u < 1e30f) corr = __fdividef(q - (u - 1.f), u);
    } else {
        u = num * rden;
    }
    const float l = logf(u) + corr;
    return l != l ? 0.f : fminf(fmaxf(l, -kLamClamp), kLamClamp);
}

// Messages of one tile.  In: nv[k] = nu (finite), lo[k] = cavity log-odds L for
// this thread's KT edges; vmask marks the edges that belong to the tile, hbits
// / tbits the ray starts / ends among them.  Out: nv[k] = lambda (valid edges).
// s_fw and s_bw hold 2 * kThreads / 32 entries each.  mid() is called by every
// thread between the CTA-wide scans and the final passes.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

template <int KT, typename Mid = NoHook>
__device__ __forceinline__ void tile_messages(float (&nv)[KT], float (&lo)[KT], uint32_t vmask, uint32_t hbits,
                                              uint32_t tbits, float nu_bg, Fwd *s_fw, Bwd *s_bw,
                                              const Mid &mid = Mid()) {
    // edges outside the tile get L = -inf, i.e. m1 = 0, m0 = 1: neutral in
    // every recurrence (their nu is any finite value)
    float c[KT], m0[KT], m1[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const float L = ((vmask >> k) & 1u) ? lo[k] : -INFINITY;
        // m = sigmoid(+-L): the approximate exp errs relative to a value it
        // then multiplies, so the probabilities keep an absolute error of a few
        // 1e-8
        const float ex = __expf(-fabsf(L));
        const float rr = recip_1_2(1.f + ex);
        const float small = ex * rr;
        m1[k] = L >= 0.f ? rr : small;
        m0[k] = L >= 0.f ? small : rr;
        c[k] = m1[k] * nv[k];
    }
    // thread aggregates (a thread holds few edges; long rays are joined by the
    // CTA-wide scans, whose combination tree keeps rounding growth logarithmic)
    Fwd fa = {0.f, 1.f, 0};
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if ((hbits >> k) & 1u) fa = {0.f, 1.f, 1};
        fa.x = fmaf(fa.y, c[k], fa.x);
        fa.y = step_P(fa.y, m0[k], m1[k]);
    }
    Bwd ba = {0.f, 1.f, 0};
#pragma unroll
    for (int k = KT - 1; k >= 0; --k) {
        if ((tbits >> k) & 1u) ba = {nu_bg, 0.f, 1};
        ba.u = step_B(ba.u, m0[k], m1[k], c[k], nv[k]);
        ba.v = step_P(ba.v, m0[k], m1[k]);
    }
    const Fwd fin = block_fwd_exclusive(fa, s_fw);
    const Bwd bin = block_bwd_exclusive(ba, s_bw);
    mid();   // all threads: a point where the caller may overlap other work
    // B_i (exclusive suffix state) for every edge, into lo[]
    float B = fmaf(bin.v, nu_bg, bin.u);
#pragma unroll
    for (int k = KT - 1; k >= 0; --k) {
        if ((tbits >> k) & 1u) B = nu_bg;
        lo[k] = B;
        B = step_B(B, m0[k], m1[k], c[k], nv[k]);
    }
    // forward pass and the messages, into nv[]
    float X = fin.x, Y = fin.y;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if ((hbits >> k) & 1u) {
            X = 0.f;
            Y = 1.f;
        }
        const float l = message(X, Y, nv[k], lo[k]);
        X = fmaf(Y, c[k], X);
        Y = step_P(Y, m0[k], m1[k]);
        nv[k] = l;
    }
}

// Bit k set for the edges my0 + k in [E0, E1).
template <int KT>
__device__ __forceinline__ uint32_t valid_mask(int64_t my0, int64_t E0, int64_t E1) {
    int64_t a = E0 - my0, b = E1 - my0;
    a = a < 0 ? 0 : (a > KT ? KT : a);
    b = b < 0 ? 0 : (b > KT ? KT : b);
    const uint32_t hi = b >= 32 ? 0xffffffffu : ((1u << (uint32_t)b) - 1u);
    const uint32_t lo = a >= 32 ? 0xffffffffu : ((1u << (uint32_t)a) - 1u);
    return hi & ~lo;
}

}  // namespace tile
}  // namespace mrf
