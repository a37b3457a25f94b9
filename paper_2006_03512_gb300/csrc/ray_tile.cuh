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
// The kernels carry these as excesses over a constant c (the likelihood
// floor: no nu and not nu_bg is below it).  With nu'_i = nu_i - c, the sums
// sum_{j<i} m1_j P_j = 1 - P_i and sum_{j>i} m1_j prod_{i<k<j} m0_k +
// prod_{k>i} m0_k = 1 give
//   A_i = c (1 - P_i) + A'_i,   A'_i = sum_{j<i} m1_j nu'_j P_j
//   B_i = c + beta_i,           beta_i = sum_{j>i} m1_j nu'_j prod_{i<k<j} m0_k
//                                        + (nu_bg - c) prod_{k>i} m0_k
// so pos_i = c + A'_i + P_i nu'_i and neg_i = c + A'_i + P_i beta_i, sums of
// non-negative terms.  On a stretch of free space whose likelihoods all sit at
// the floor (= nu_bg by default), nu', A' and beta are exactly zero and so is
// the message; computed directly, B would drift from nu_bg by rounding
// (m1 + m0 is not exactly 1 in FP32) and leave messages of a few 1e-7 that add
// up, with one sign, over the many rays crossing a voxel near the camera.
//
// A' and P are a forward linear recurrence, (A', P) <- (A' + P m1 nu', P m0);
// beta is a backward one, beta <- m1 nu' + m0 beta, started at nu_bg - c after
// a ray's last voxel.  Every quantity stays bounded: P is a probability, and
// A' and beta are sums of likelihood excesses weighted by probabilities.  So both
// scans run in plain FP32 without log-domain rescaling; the transcendentals
// per edge are one exp and one reciprocal (for m1, m0) and one reciprocal and
// one log (for lambda).
//
// A tile is a run of whole rays; each of the CTA's 256 threads holds KT
// consecutive edges, scans them sequentially, and the CTA combines the
// thread aggregates with warp shuffles (segmented by ray starts and ends).
#pragma once

#include "mrf_internal.cuh"

namespace mrf {
namespace tile {

// Forward map (A, P) -> (A + x P, |y| P); a map that starts a ray (resets the
// state first) carries the sign bit of y.  Every factor of y is >= 0 and no
// step cancels it exactly, so the sign bit survives the products.
struct Fwd {
    float x, y;
};
// Backward map B -> u + v B.  A map that contains a ray end is constant: v = 0
// exactly, and composing with it keeps v = 0 and u unchanged.
struct Bwd {
    float u, v;
};

__device__ __forceinline__ bool starts_ray(const Fwd &a) { return __float_as_int(a.y) < 0; }

__device__ __forceinline__ Fwd fwd_op(const Fwd &a, const Fwd &b) {  // a precedes b
    if (starts_ray(b)) return b;
    return {fmaf(fabsf(a.y), b.x, a.x), a.y * fabsf(b.y)};
}
__device__ __forceinline__ Bwd bwd_op(const Bwd &lo, const Bwd &hi) {  // hi is applied first
    return {fmaf(lo.v, hi.u, lo.u), lo.v * hi.v};
}
__device__ __forceinline__ Fwd shfl_up(const Fwd &a, int o) {
    return {__shfl_up_sync(0xffffffffu, a.x, o), __shfl_up_sync(0xffffffffu, a.y, o)};
}
__device__ __forceinline__ Bwd shfl_down(const Bwd &a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.u, o), __shfl_down_sync(0xffffffffu, a.v, o)};
}
__device__ __forceinline__ Fwd shfl_idx(const Fwd &a, int l) {
    return {__shfl_sync(0xffffffffu, a.x, l), __shfl_sync(0xffffffffu, a.y, l)};
}
__device__ __forceinline__ Bwd shfl_idx(const Bwd &a, int l) {
    return {__shfl_sync(0xffffffffu, a.u, l), __shfl_sync(0xffffffffu, a.v, l)};
}

// Exclusive forward (prefix) and backward (suffix) scans over the CTA's
// threads, together: warps scan with shuffles and publish their totals; after
// one barrier every warp scans the 8 totals itself and takes its own prefix
// and suffix.  NT threads; s_fw and s_bw need NT / 32 entries; they are read
// until the caller's next barrier.
template <int NT = kThreads>
__device__ __forceinline__ void block_scans(Fwd fv, Bwd bv, Fwd *s_fw, Bwd *s_bw, Fwd &fin, Bwd &bin) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Fwd fid = {0.f, 1.f};
    const Bwd bid = {0.f, 1.f};
    Fwd fi = fv;
    Bwd bi = bv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Fwd y = shfl_up(fi, o);
        const Bwd z = shfl_down(bi, o);
        if (lane >= o) fi = fwd_op(y, fi);
        if (lane + o < 32) bi = bwd_op(bi, z);
    }
    Fwd fex = shfl_up(fi, 1);
    Bwd bex = shfl_down(bi, 1);
    if (lane == 0) fex = fid;
    if (lane == 31) bex = bid;
    if (lane == 31) s_fw[warp] = fi;
    if (lane == 0) s_bw[warp] = bi;
    __syncthreads();
    Fwd ft = lane < NW ? s_fw[lane] : fid;
    Bwd bt = lane < NW ? s_bw[lane] : bid;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const Fwd y = shfl_up(ft, o);
        const Bwd z = shfl_down(bt, o);
        if (lane >= o) ft = fwd_op(y, ft);
        if (lane + o < NW) bt = bwd_op(bt, z);
    }
    Fwd fp = shfl_idx(ft, (warp + 31) & 31);   // inclusive over warps < warp
    Bwd bs = shfl_idx(bt, (warp + 1) & 31);    // inclusive over warps > warp
    if (warp == 0) fp = fid;
    if (warp == NW - 1) bs = bid;
    fin = fwd_op(fp, fex);
    bin = bwd_op(bex, bs);
}

// One step of the visibility product, P <- P m0, and of the backward state,
// B <- m1 nu + m0 B = B + m1 (nu - B).  A free-space voxel has m0 = 1 - m1 with
// m1 tiny, and m0 stored in FP32 keeps only a few digits of m1; so when m1 < 1/2
// the steps are taken through m1 (P - m1 P and (B + c) - m1 B, c = m1 nu), and
// through m0 otherwise (where m0 is the small, precise one).  Both forms are
// P <- alpha P + beta P and B <- alpha B + (beta B + c) with, per edge,
// (alpha, beta) = (-m1, 1) or (m0, 0), so the steps need no branch or select.
__device__ __forceinline__ float step_P(float P, float a, float b) { return fmaf(a, P, b * P); }
__device__ __forceinline__ float step_B(float B, float a, float b, float c) { return fmaf(a, B, fmaf(b, B, c)); }

// 1/x to about 1 ulp for x in [1e-30, 1e30]: the hardware reciprocal estimate
// refined by one Newton step (outside that range, where the estimate flushes,
// the correctly rounded reciprocal).
__device__ __forceinline__ float recip(float x) {
    if (!(x > 1e-30f && x < 1e30f)) return __frcp_rn(x);
    const float r = __fdividef(1.f, x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// The same for x in [1e-30, 1e30] known in advance (no range test).
__device__ __forceinline__ float recip_in_range(float x) {
    const float r = __fdividef(1.f, x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// The same for x in [1, 2], where the estimate never flushes.
__device__ __forceinline__ float recip_1_2(float x) {
    const float r = __fdividef(1.f, x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// lambda = log(pos / neg) from pos = c + A' + P nu' and
// neg = c + A' + P beta (the excess form above).  With
// q = (pos - neg) / neg = P (nu' - beta) / neg, log(1 + q) is formed as
// log(u) + (q - (u - 1)) / u with u = fl(1 + q), which keeps full relative
// precision for the many near-zero messages; where q <= -1/2 (pos well below
// neg) 1 + q would lose bits and u = pos / neg, a ratio of two non-negative
// sums, is used directly.  neg = 0 (possible only when nu_bg = 0) gives +64, or
// 0 when pos is 0 as well.
// FL ("floored"): the caller guarantees 1e-30 <= c0 and every nu below 1e29 and
// below 1e25 c0.  Then c0 <= neg < 1e30 and |lambda| < 58, so the tests for
// neg = 0, the reciprocal's range, NaN and the clamp are all dead and left out.
template <bool FL = false>
__device__ __forceinline__ float message(float Ax, float P, float nux, float beta, float c0) {
    const float base = Ax + c0;
    const float num = fmaf(P, nux, base);
    const float den = fmaf(P, beta, base);
    if (!FL && !(den > 0.f)) return num > 0.f ? kLamClamp : 0.f;
    const float rden = FL ? recip_in_range(den) : recip(den);
    const float q = P * (nux - beta) * rden;
    float u, corr = 0.f;
    if (q > -0.5f) {
        u = 1.f + q;
        if (FL || u < 1e30f) corr = __fdividef(q - (u - 1.f), u);
    } else {
        u = num * rden;
    }
    const float l = logf(u) + corr;
    if (FL) return l;
    return l != l ? 0.f : fminf(fmaxf(l, -kLamClamp), kLamClamp);
}

// Messages of one tile.  In: nv[k] = nu (finite), lo[k] = cavity log-odds L for
// this thread's KT edges; vmask marks the edges that belong to the tile, hbits
// / tbits the ray starts / ends among them; nu_ref = c <= min(nu, nu_bg) (0
// always qualifies).  Out: nv[k] = lambda (valid edges).
// s_fw and s_bw hold NT / 32 entries each (NT threads).  mid() is called by every
// thread between the CTA-wide scans and the final passes.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

template <int KT, int NT = kThreads, bool FL = false, typename Mid = NoHook>
__device__ __forceinline__ void tile_messages(float (&nv)[KT], float (&lo)[KT], uint32_t vmask, uint32_t hbits,
                                              uint32_t tbits, float nu_bg, float nu_ref, Fwd *s_fw,
                                              Bwd *s_bw, const Mid &mid = Mid()) {
    const float bg_x = nu_bg - nu_ref;   // beta after a ray's last voxel
    // edges outside the tile get L = -inf, i.e. m1 = 0, m0 = 1: neutral in
    // every recurrence (their nu is any finite value)
    float c[KT], al[KT], be[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const float L = ((vmask >> k) & 1u) ? lo[k] : -INFINITY;
        // m = sigmoid(+-L): the approximate exp errs relative to a value it
        // then multiplies, so the probabilities keep an absolute error of a few
        // 1e-8.  small = min(m0, m1); m1 < 1/2 exactly when L < 0.
        const float ex = __expf(-fabsf(L));
        const float rr = recip_1_2(1.f + ex);
        const float small = ex * rr;
        const bool neg = L < 0.f;
        al[k] = neg ? -small : small;
        be[k] = neg ? 1.f : 0.f;
        nv[k] -= nu_ref;   // nu': zero where nu is at the floor
        c[k] = (neg ? small : rr) * nv[k];
    }
    // thread aggregates (a thread holds few edges; long rays are joined by the
    // CTA-wide scans, whose combination tree keeps rounding growth logarithmic)
    Fwd fa = {0.f, 1.f};
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if ((hbits >> k) & 1u) fa = {0.f, -1.f};   // starts a ray: sign bit set
        fa.x = fmaf(fabsf(fa.y), c[k], fa.x);
        fa.y = step_P(fa.y, al[k], be[k]);          // keeps the sign
    }
    Bwd ba = {0.f, 1.f};
#pragma unroll
    for (int k = KT - 1; k >= 0; --k) {
        if ((tbits >> k) & 1u) ba = {bg_x, 0.f};
        ba.u = step_B(ba.u, al[k], be[k], c[k]);
        ba.v = step_P(ba.v, al[k], be[k]);
    }
    Fwd fin;
    Bwd bin;
    block_scans<NT>(fa, ba, s_fw, s_bw, fin, bin);
    mid();   // all threads: a point where the caller may overlap other work
    // beta_i (exclusive suffix state) for every edge, into lo[]; a tile ends
    // with a ray end
    float B = fmaf(bin.v, bg_x, bin.u);
#pragma unroll
    for (int k = KT - 1; k >= 0; --k) {
        if ((tbits >> k) & 1u) B = bg_x;
        lo[k] = B;
        B = step_B(B, al[k], be[k], c[k]);
    }
    // forward pass and the messages, into nv[]
    float X = fin.x, Y = fabsf(fin.y);
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if ((hbits >> k) & 1u) {
            X = 0.f;
            Y = 1.f;
        }
        const float l = message<FL>(X, Y, nv[k], lo[k], nu_ref);
        X = fmaf(Y, c[k], X);
        Y = step_P(Y, al[k], be[k]);
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
