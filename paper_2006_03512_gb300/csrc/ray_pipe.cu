// Ray -> voxel messages for the context's own (padded) edge arrays: a
// persistent, software-pipelined version of the per-tile computation in
// ray_tile.cuh.
//
// Each CTA owns a contiguous range of ray tiles (neighbouring rays, so their
// voxels and the T entries they gather overlap).  Two shared-memory stages
// hold a tile's likelihoods, old messages, group (or voxel) indices, window
// indices, the window's ray-start and group-end bitmap words and its group
// keys; the next tile's stage is filled by TMA bulk copies (cp.async.bulk,
// completion on an mbarrier) issued when the current tile starts.  Half-way
// through the current tile (once the thread aggregates are published) the
// threads wait for that copy, and the threads of warps 2 and up gather the
// next tile's voxel totals with cp.async, one per (tile, voxel) group (per
// window position without grouping); those land while the current tile
// finishes.  Two stages keep shared memory at ~74 KB, so three CTAs fit on
// an SM.
//
// The kernel is bound by latency (its gathers' L1/shared-memory traffic and
// its barriers) and instruction issue, not by HBM, so its arithmetic is
// written for few instructions per edge:
//   * the CTA-wide scans combine the 256 thread aggregates in two warps
//     (forward and backward), by a tree over 8 aggregates per lane and by
//     shuffles across lanes, while the other warps gather the next tile;
//   * the per-edge coefficient and message arithmetic runs on pairs of edges
//     with Blackwell's paired FP32 instructions (__fadd2_rn, __fmul2_rn,
//     __ffma2_rn), one issue slot for two edges;
//   * in the floored form the forward recurrence is carried as one affine
//     state (the odds form below), and every thread keeps its local forward
//     and backward maps in front of each edge: after the CTA scans each edge's
//     states are one FMA away, with no second pass over the ray starts and ends;
//   * the message log uses lambda = 2 atanh(s), s = (num - den) / (num + den),
//     by its odd series where |s| <= 1/4 and ln 2 log2(num / den) elsewhere;
//   * gathers and the per-edge arithmetic run unmasked; only the one thread at
//     each end of a tile, whose slice reaches outside the tile, masks its
//     positions (cavity -inf: m1 = 0, neutral in every recurrence);
//   * per tile, each thread's bounds and bitmap shifts are 32-bit offsets
//     within the window.
//
// Every mbarrier wait is bounded; a wait that gives up sets bit 1 of *err, and
// the CTA leaves after all threads agree (no thread is left at a barrier).
#include <cuda_bf16.h>

#include <cstddef>
#include <type_traits>

#include "async_copy.cuh"
#include "mrf_internal.cuh"
#include "ray_tile.cuh"

namespace mrf {
namespace {

using tile::Bwd;
using tile::Fwd;

using async::cp_async4;
using async::cp_async_commit;
using async::cp_async_wait;
using async::mbar_expect_tx;
using async::mbar_init;
using async::mbar_wait;
using async::smem_u32;
using async::tma_load_1d;

// Per-edge messages are stored as FP32, or as bf16 (rounded to nearest even;
// the arithmetic is FP32 either way).
template <typename LamT>
__host__ __device__ constexpr bool is_bf16() { return std::is_same<LamT, __nv_bfloat16>::value; }

// Shared memory of one CTA.  Two stages (tiles j and j + 1) of the per-edge
// inputs; the scans' aggregates and the epilogue's tails are single buffers,
// rewritten only after every thread has passed the previous tile's barriers.
// With grouping (AGG) the voxel totals are gathered once per (tile, voxel)
// group into T and read through each edge's group index (gid); without it,
// once per edge through the voxel keys (vox).  nu[st] holds the tile's
// messages by window index for the grouping epilogue (each thread writes only
// the positions whose likelihoods it read itself); thread 0 refills it when it
// starts tile j + 1, after the epilogue's last barrier.
template <int KT, int NT, typename LamT, bool AGG>
struct PipeSmem {
    static constexpr int CAP = NT * KT;
    static constexpr int NA = NT + NT / 8;   // aggregates, one float2 of padding per 8 (bank spread)
    // every array starts on a 16-byte boundary: bulk copies, cp.async and the
    // vector loads need it, and the placeholders of the unused arrays are small
    alignas(16) float nu[2][CAP];         // likelihoods; then the tile's messages by window index
    alignas(16) LamT lam[2][CAP];
    // gathered voxel totals: per window position, or (AGG) per group, slot g at
    // g + toff (the groups' keys arrive by a bulk copy from a 16-byte boundary)
    alignas(16) float T[2][CAP + 8];
    alignas(16) uint32_t vox[AGG ? 1 : 2][AGG ? 1 : CAP];   // voxel keys (without grouping)
    alignas(16) uint16_t gid[AGG ? 2 : 1][AGG ? CAP : 1];   // group of each window position (grouping)
    alignas(16) uint16_t lx[AGG ? 2 : 1][AGG ? CAP : 1];    // window index of each tile-major position (grouping)
    // the ray-start (hb) and group-end (eb, grouping) bitmap words covering the
    // window, from the 16-byte boundary at or below its first word
    static constexpr int KW = CAP / 32 + 4;
    alignas(16) uint32_t hb[2][KW];
    alignas(16) uint32_t eb[AGG ? 2 : 1][AGG ? KW : 4];
    alignas(16) float2 fagg[NA];                 // thread aggregates, then exclusive prefixes (forward)
    alignas(16) float2 bagg[NA];                 // the same for the backward scan (suffixes)
    alignas(16) float2 tail[AGG ? NT : 1];   // per thread: sum after its last group end, and whether it has one
    int64_t E0[2], E1[2], tg[2], tge[2];
    int toff[2];
    int64_t nE0, nE1, ntg, ntge;   // the tile after the next one's range and slots, prefetched
    uint64_t bar[2];
};
template <int KT, int NT, typename LamT, bool AGG>
__host__ __device__ constexpr bool pipe_smem_aligned() {
    using S = PipeSmem<KT, NT, LamT, AGG>;
    return offsetof(S, nu) % 16 == 0 && offsetof(S, lam) % 16 == 0 && offsetof(S, T) % 16 == 0 &&
           offsetof(S, vox) % 16 == 0 && offsetof(S, gid) % 16 == 0 && offsetof(S, lx) % 16 == 0 &&
           sizeof(((S *)0)->nu[0]) % 16 == 0 && sizeof(((S *)0)->lam[0]) % 16 == 0;
}

// Bit k set for k in [a, b) (0 <= k < KT), from window-relative bounds.
template <int KT>
__device__ __forceinline__ uint32_t valid_mask32(int a, int b) {
    a = min(max(a, 0), KT);
    b = min(max(b, 0), KT);
    const uint32_t hi = b >= 32 ? 0xffffffffu : ((1u << (uint32_t)b) - 1u);
    const uint32_t lo = a >= 32 ? 0xffffffffu : ((1u << (uint32_t)a) - 1u);
    return hi & ~lo;
}

// First edge of a tile's 256*KT-edge window (aligned to 8 edges).
__device__ __forceinline__ int64_t window_base(int64_t E0) { return E0 & ~(int64_t)7; }

// Resident CTAs per SM the register budget is set for: three for 2048-edge
// tiles (about 76 KB of shared memory each), one otherwise.
template <int KT, int NT>
constexpr int pipe_min_blocks() { return NT * KT == 2048 ? (NT >= 512 ? 2 : 3) : 1; }

// ---- paired FP32 arithmetic (one instruction for two lanes' worth of work)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

// hardware reciprocal and base-2 logarithm estimates (about one ulp; inputs
// here are normal numbers)
__device__ __forceinline__ float rcp_est(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_est(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-edge coefficients of the recurrences (ray_tile.cuh) for two edges of
// cavity log-odds L: with e = exp(-|L|) and r = 1 / (1 + e), the larger of
// m1 = sigmoid(L), m0 = sigmoid(-L) is r and the smaller e r.  al, be are the
// step coefficients (P <- al P + be P), c = m1 (nu - nu_ref).
__device__ __forceinline__ void coeff_pair(float2 L, float2 &nux, float nu_ref, float2 &al, float2 &be, float2 &c) {
    const float2 e = make_float2(__expf(-fabsf(L.x)), __expf(-fabsf(L.y)));
    const float2 w = add2(e, splat(1.f));
    const float2 r = make_float2(rcp_est(w.x), rcp_est(w.y));
    const float2 sm = mul2(e, r);
    const bool n0 = L.x < 0.f, n1 = L.y < 0.f;
    al = make_float2(n0 ? -sm.x : sm.x, n1 ? -sm.y : sm.y);
    be = make_float2(n0 ? 1.f : 0.f, n1 ? 1.f : 0.f);
    const float2 m1 = make_float2(n0 ? sm.x : r.x, n1 ? sm.y : r.y);
    nux = add2(nux, splat(-nu_ref));
    c = mul2(m1, nux);
}

// ---- the odds form of the forward recurrence (floored kernels)
//
// With t_i = exp(L_i) = m1_i / m0_i (the cavity odds) and R_i = (c + A'_i) / P_i,
// the forward pair (A', P) of ray_tile.cuh becomes one affine recurrence,
//   R_{i+1} = (R_i + m1_i nu'_i) / m0_i = R_i + t_i (R_i + nu'_i),   R = c at a ray start,
// and dividing pos_i and neg_i by P_i gives lambda_i = log((R_i + nu'_i) / (R_i + beta_i)).
// Each step rounds once relative to R, as the visibility product does in the
// (A', P) form, and on free space at the likelihood floor (nu' = beta = 0) the
// message is still exactly 0.  A thread composes its edges' maps R -> a + b R
// (b = 0 from a ray start on) and keeps the map in front of every edge, so
// that once the CTA scan hands it the state at its first edge each R_i is one
// FMA with no test of the ray starts; the backward maps beta -> u + v beta are
// kept the same way.
//
// R grows where the visibility P vanishes.  Cavities are clamped at 80 before
// the exponential and t is raised by 1e-30, so t is finite and positive (no
// 0 * inf in a step; the 1e-30 is far below the rounding of every state it
// meets), and the thread aggregates and their compositions are clamped at
// FLT_MAX; an R that large (or infinite) gives num = den = inf and s = 0, i.e.
// a zero message, the limit of the exact one.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kOddsLmax = 80.f;
constexpr float kRmax = 3.402823466e38f;   // FLT_MAX

// The forward state and per-edge maps of the odds form: R -> a + b R.
struct Aff {
    float a, b;
};
// p then q, clamped (inputs <= FLT_MAX and >= 0, so no 0 * inf)
__device__ __forceinline__ Aff aff_op(const Aff &p, const Aff &q) {
    return {fminf(fmaf(q.b, p.a, q.a), kRmax), fminf(q.b * p.b, kRmax)};
}

// Per-edge coefficients for the odds form, two edges at a time: t = exp(L)
// (L clamped at 80, t raised by 1e-30), and the backward recurrence's al, be, c = m1 nu' as in
// coeff_pair (m1 = t r, m0 = r with r = 1 / (1 + t); the smaller of the two is
// the one the step is taken through).
__device__ __forceinline__ void coeff_odds(float2 L, float2 &nux, float nu_ref, float2 &t, float2 &al, float2 &be,
                                           float2 &c) {
    const float2 Lc = make_float2(fminf(L.x, kOddsLmax), fminf(L.y, kOddsLmax));
    const float2 x = mul2(Lc, splat(kLog2e));
    float2 e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(x.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(x.y));
    e = add2(e, splat(1e-30f));
    t = e;
    const float2 w = add2(e, splat(1.f));
    const float2 r = make_float2(rcp_est(w.x), rcp_est(w.y));
    const float2 m1 = mul2(e, r);
    const bool n0 = L.x < 0.f, n1 = L.y < 0.f;
    al = make_float2(n0 ? -m1.x : r.x, n1 ? -m1.y : r.y);
    be = make_float2(n0 ? 1.f : 0.f, n1 ? 1.f : 0.f);
    nux = add2(nux, splat(-nu_ref));
    c = mul2(m1, nux);
}

// Messages of two edges in the odds form: num = R + nu', den = R + beta (pos and
// neg over the visibility), lambda = log(num / den) = 2 atanh(s) with
// s = (num - den) / (num + den) = (nu' - beta) / (num + den), formed without
// cancellation.  For |s| <= 1/4 (|lambda| <= 0.51) the odd series
// 2 (s + s^3/3 + ... + s^11/11) is used: its truncation is below 5e-9 relative,
// so the many near-zero messages keep full relative precision.  Otherwise
// lambda = ln 2 log2(num / den), whose absolute error (about 1e-7) is below
// 3e-7 of such a message.  R = inf (or num + den = inf) gives s = 0 and lambda = 0.
__device__ __forceinline__ float2 message_pair_odds(float2 R, float2 nux, float2 beta) {
    const float2 num = add2(R, nux);
    const float2 den = add2(R, beta);
    const float2 D = fma2(beta, splat(-1.f), nux);
    const float2 sum = add2(num, den);
    const float2 s = mul2(D, make_float2(rcp_est(sum.x), rcp_est(sum.y)));
    const float2 t = mul2(s, s);
    float2 q = fma2(t, splat(2.f / 11.f), splat(2.f / 9.f));
    q = fma2(t, q, splat(2.f / 7.f));
    q = fma2(t, q, splat(2.f / 5.f));
    q = fma2(t, q, splat(2.f / 3.f));
    q = fma2(t, q, splat(2.f));
    const float2 ls = mul2(s, q);
    const float2 u = mul2(num, make_float2(rcp_est(den.x), rcp_est(den.y)));
    const float2 ll = mul2(make_float2(lg2_est(u.x), lg2_est(u.y)), splat(0.6931471805599453f));
    return make_float2(fabsf(s.x) <= 0.25f ? ls.x : ll.x, fabsf(s.y) <= 0.25f ? ls.y : ll.y);
}

// The CTA-wide exclusive scans of the thread aggregates.  Every thread has
// published its forward aggregate in s_f and backward aggregate in s_b (index
// agg_slot(tid)) before a barrier; then warp 0 turns s_f into exclusive
// prefixes and warp 1 turns s_b into exclusive suffixes.  Each lane combines
// NT/32 consecutive aggregates into its total by a tree of pairs (a chain of
// log2(NT/32) compositions instead of NT/32), the lanes' totals are scanned by
// shuffles, and each lane then writes its exclusive prefixes: with eight
// aggregates per lane from the pair sums kept by the tree (three compositions
// deep), otherwise sequentially.  The results are read after the next barrier.
// The sequential loops are unrolled only by two: the thread's per-edge arrays
// are live across this code.
template <int NA, int NT>
__device__ __forceinline__ int agg_slot(int t) { return t + (t >> 3); }

template <int NT, int NA>
__device__ __forceinline__ void scan_fwd_warp(float2 *s_f) {
    constexpr int PER = NT / 32;
    const int lane = threadIdx.x & 31;
    const Fwd fid = {0.f, 1.f};
    Fwd tot = fid;
#pragma unroll 2
    for (int j = 0; j < PER; ++j) {
        const float2 a = s_f[agg_slot<NA, NT>(lane * PER + j)];
        tot = tile::fwd_op(tot, Fwd{a.x, a.y});
    }
    Fwd inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Fwd y = tile::shfl_up(inc, o);
        if (lane >= o) inc = tile::fwd_op(y, inc);
    }
    Fwd run = tile::shfl_up(inc, 1);
    if (lane == 0) run = fid;
#pragma unroll 2
    for (int j = 0; j < PER; ++j) {
        const int i = agg_slot<NA, NT>(lane * PER + j);
        const float2 a = s_f[i];
        s_f[i] = make_float2(run.x, run.y);
        run = tile::fwd_op(run, Fwd{a.x, a.y});
    }
}

// The same exclusive prefix scan for the odds form's maps R -> a + b R.
template <int NT, int NA>
__device__ __forceinline__ void scan_fwd_warp_odds(float2 *s_f) {
    constexpr int PER = NT / 32;
    const int lane = threadIdx.x & 31;
    const Aff fid = {0.f, 1.f};
    Aff v[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const float2 a = s_f[agg_slot<NA, NT>(lane * PER + j)];
        v[j] = Aff{a.x, a.y};
    }
    Aff m01 = fid, m45 = fid, m0123 = fid;   // pair sums kept for the write-back (PER == 8)
#pragma unroll
    for (int w = 1; w < PER; w <<= 1) {
#pragma unroll
        for (int j = 0; j + w < PER; j += 2 * w) v[j] = aff_op(v[j], v[j + w]);
        if (PER == 8 && w == 1) {
            m01 = v[0];
            m45 = v[4];
        }
        if (PER == 8 && w == 2) m0123 = v[0];
    }
    Aff tot = v[0];
    Aff inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Aff y = {__shfl_up_sync(0xffffffffu, inc.a, o), __shfl_up_sync(0xffffffffu, inc.b, o)};
        if (lane >= o) inc = aff_op(y, inc);
    }
    Aff run = {__shfl_up_sync(0xffffffffu, inc.a, 1), __shfl_up_sync(0xffffffffu, inc.b, 1)};
    if (lane == 0) run = fid;
    if constexpr (PER == 8) {
        // exclusive prefixes from the kept pair sums: depth three instead of eight
        auto ld = [&](int j) {
            const float2 a = s_f[agg_slot<NA, NT>(lane * PER + j)];
            return Aff{a.x, a.y};
        };
        auto st = [&](int j, const Aff &p) { s_f[agg_slot<NA, NT>(lane * PER + j)] = make_float2(p.a, p.b); };
        const Aff a0 = ld(0), a2 = ld(2), a4 = ld(4), a6 = ld(6);
        const Aff p2 = aff_op(run, m01), p4 = aff_op(run, m0123);
        const Aff p6 = aff_op(p4, m45);
        st(0, run);
        st(1, aff_op(run, a0));
        st(2, p2);
        st(3, aff_op(p2, a2));
        st(4, p4);
        st(5, aff_op(p4, a4));
        st(6, p6);
        st(7, aff_op(p6, a6));
    } else {
#pragma unroll 2
        for (int j = 0; j < PER; ++j) {
            const int i = agg_slot<NA, NT>(lane * PER + j);
            const float2 a = s_f[i];
            s_f[i] = make_float2(run.a, run.b);
            run = aff_op(run, Aff{a.x, a.y});
        }
    }
}

template <int NT, int NA>
__device__ __forceinline__ void scan_bwd_warp(float2 *s_b) {
    constexpr int PER = NT / 32;
    const int lane = threadIdx.x & 31;
    const Bwd bid = {0.f, 1.f};
    Bwd v[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const float2 a = s_b[agg_slot<NA, NT>(lane * PER + j)];
        v[j] = Bwd{a.x, a.y};
    }
#pragma unroll
    for (int w = 1; w < PER; w <<= 1)
#pragma unroll
        for (int j = 0; j + w < PER; j += 2 * w) v[j] = tile::bwd_op(v[j], v[j + w]);
    Bwd tot = v[0];
    Bwd inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Bwd z = tile::shfl_down(inc, o);
        if (lane + o < 32) inc = tile::bwd_op(inc, z);
    }
    Bwd run = tile::shfl_down(inc, 1);
    if (lane == 31) run = bid;
    if constexpr (PER == 8) {
        // exclusive suffixes from the pair sums the up-sweep left in v[2]
        // (a2 a3), v[6] (a6 a7) and v[4] (a4 .. a7): depth three instead of eight
        auto ld = [&](int j) {
            const float2 a = s_b[agg_slot<NA, NT>(lane * PER + j)];
            return Bwd{a.x, a.y};
        };
        auto st = [&](int j, const Bwd &p) { s_b[agg_slot<NA, NT>(lane * PER + j)] = make_float2(p.u, p.v); };
        const Bwd a1 = ld(1), a3 = ld(3), a5 = ld(5), a7 = ld(7);
        const Bwd s5 = tile::bwd_op(v[6], run), s3 = tile::bwd_op(v[4], run);
        const Bwd s1 = tile::bwd_op(v[2], s3);
        st(7, run);
        st(6, tile::bwd_op(a7, run));
        st(5, s5);
        st(4, tile::bwd_op(a5, s5));
        st(3, s3);
        st(2, tile::bwd_op(a3, s3));
        st(1, s1);
        st(0, tile::bwd_op(a1, s1));
    } else {
#pragma unroll 2
        for (int j = PER - 1; j >= 0; --j) {
            const int i = agg_slot<NA, NT>(lane * PER + j);
            const float2 a = s_b[i];
            s_b[i] = make_float2(run.u, run.v);
            run = tile::bwd_op(Bwd{a.x, a.y}, run);
        }
    }
}

template <int KT, bool AGG, int NT, typename LamT, bool FL>
__global__ void __launch_bounds__(NT, pipe_min_blocks<KT, NT>())
    k_ray_pipe(const int64_t *__restrict__ tile_E, int64_t ntiles, const uint32_t *__restrict__ hb,
               const uint32_t *__restrict__ vox, const float *__restrict__ nu, const float *__restrict__ T,
               LamT *__restrict__ lam, float nu_bg, float nu_ref, int first, float L0, uint32_t *__restrict__ err,
               const uint16_t *__restrict__ lidx, const uint32_t *__restrict__ ends,
               const uint16_t *__restrict__ gid, const uint32_t *__restrict__ gkey,
               const int64_t *__restrict__ tg_off, float *__restrict__ partial) {
    static_assert(KT % 4 == 0, "a thread's edges are loaded four at a time");
    using S = PipeSmem<KT, NT, LamT, AGG>;
    static_assert(pipe_smem_aligned<KT, NT, LamT, AGG>(), "bulk-copy destinations on 16-byte boundaries");
    constexpr int CAP = S::CAP;
    constexpr int KP = KT / 2;   // edge pairs per thread
    extern __shared__ __align__(128) uint8_t smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * ntiles / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * ntiles / gridDim.x;
    const int n = (int)(t1 - t0);
    if (n <= 0) return;
    // per stage: likelihoods and, with grouping, the group indices (the
    // epilogue numbers its groups by them) and the window index of each
    // tile-major position, and the bitmap words of the window; after the first pass also the old
    // messages and, without grouping, the voxel keys (with grouping, the
    // groups' keys, whose size varies by tile, are added in issue())
    const uint32_t stage_bytes = (uint32_t)(CAP * 4) + (AGG ? (uint32_t)(CAP * 4) : 0u) +
                                 (uint32_t)(S::KW * 4 * (AGG ? 2 : 1)) +
                                 (first ? 0u : (uint32_t)(CAP * (sizeof(LamT) + (AGG ? 0 : 4))));

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) mbar_init(&sm.bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0: bulk copies of tile j into stage j % 2 (tile j's range and
    // first slot: loaded for tile 0, else prefetched by the gathers of tile j - 1)
    auto issue = [&](int j) {
        const int st = j & 1;
        const int64_t E0 = j ? sm.nE0 : tile_E[t0 + j], E1 = j ? sm.nE1 : tile_E[t0 + j + 1];
        const int64_t base = window_base(E0);
        sm.E0[st] = E0;
        sm.E1[st] = E1;
        if (AGG) {
            sm.tg[st] = j ? sm.ntg : tg_off[t0 + j];
            sm.tge[st] = j ? sm.ntge : tg_off[t0 + j + 1];
        }
        // with grouping, after the first pass: the tile's group keys, copied
        // from the 16-byte boundary at or below the first one (slot g lands at
        // g + toff); each gathered total later replaces its key
        uint32_t key_bytes = 0;
        int64_t ka = 0;
        if (AGG && !first) {
            const int64_t tg0 = sm.tg[st], tg1 = sm.tge[st];
            ka = tg0 & ~(int64_t)3;
            key_bytes = (uint32_t)((((tg1 + 3) & ~(int64_t)3) - ka) * 4);
            sm.toff[st] = (int)(tg0 - ka);
        } else {
            sm.toff[st] = 0;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&sm.bar[st], stage_bytes + key_bytes);
        tma_load_1d(sm.nu[st], nu + base, CAP * 4, &sm.bar[st]);
        if (key_bytes) tma_load_1d(sm.T[st], gkey + ka, key_bytes, &sm.bar[st]);
        const int64_t wa = (base >> 5) & ~(int64_t)3;
        tma_load_1d(sm.hb[st], hb + wa, S::KW * 4, &sm.bar[st]);
        if constexpr (AGG) {
            tma_load_1d(sm.gid[st], gid + base, CAP * 2, &sm.bar[st]);
            tma_load_1d(sm.lx[st], lidx + base, CAP * 2, &sm.bar[st]);
            tma_load_1d(sm.eb[st], ends + wa, S::KW * 4, &sm.bar[st]);
        }
        if (!first) {
            if constexpr (!AGG) tma_load_1d(sm.vox[st], vox + base, CAP * 4, &sm.bar[st]);
            tma_load_1d(sm.lam[st], lam + base, CAP * (uint32_t)sizeof(LamT), &sm.bar[st]);
        }
    };
    // every thread, once tile j's bulk copy is in: cp.async of T entries (per
    // group, or per window position without grouping; the library keeps the
    // keys past the last edge valid).
    auto gather = [&](int j) {
        const int st = j & 1;
        if (tid == 0 && j + 1 < n) {   // tile j + 1's scalars, for its bulk copies when tile j starts
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.nE0)), "l"(tile_E + t0 + j + 1)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.nE1)), "l"(tile_E + t0 + j + 2)
                         : "memory");
            if (AGG) {
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.ntg)),
                             "l"(tg_off + t0 + j + 1)
                             : "memory");
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.ntge)),
                             "l"(tg_off + t0 + j + 2)
                             : "memory");
            }
        }
        if (!first) {
            if constexpr (AGG) {
                // one voxel total per group of the tile, by the threads of warps
                // 2 and up (warps 0 and 1 run the scans meanwhile); visible to the
                // CTA after the epilogue's last barrier of the current tile.  The
                // groups' keys are already in the slots (the tile's bulk copy, on
                // whose barrier every thread has waited), and each slot's total
                // replaces its key.
                const int ng = (int)(sm.tge[st] - sm.tg[st]);
                constexpr int NG = NT - 64;
                if (tid >= 64) {
                    float *Ts = sm.T[st] + sm.toff[st];
#pragma unroll 4
                    for (int g = tid - 64; g < ng; g += NG) cp_async4(&Ts[g], T + __float_as_uint(Ts[g]));
                }
            } else {
                // a warp gathers the T entries of its own threads' edges, lane l
                // taking every 32nd edge from l: neighbouring edges of a ray share
                // cache sectors, so a warp-wide gather touches fewer of them
                const int wb = (tid & ~31) * KT + (tid & 31);
#pragma unroll
                for (int k = 0; k < KT; ++k) {
                    const int i = wb + k * 32;
                    cp_async4(&sm.T[st][i], T + sm.vox[st][i]);
                }
            }
        }
        cp_async_commit();
    };

    if (tid == 0) issue(0);
    __syncthreads();
    {
        const bool ok = mbar_wait(&sm.bar[0], 0);
        if (__syncthreads_or(!ok)) {   // tile 0's copy never completed; nothing of ours is in flight
            if (tid == 0) atomicOr(err, 2u);
            return;
        }
    }
    gather(0);
    cp_async_wait<0>();
    __syncthreads();   // tile 0's gathers (by any thread) are in

    const float bg_x = nu_bg - nu_ref;   // beta after a ray's last voxel
    for (int j = 0; j < n; ++j) {
        const int st = j & 1;
        cp_async_wait<0>();   // this thread's copies for tile j (thread 0: and tile j + 1's scalars)
        if (tid == 0 && j + 1 < n) issue(j + 1);
        // the other lanes' copies: without grouping a warp gathered its own
        // edges' totals; with it every thread waited for its gathers before
        // the previous tile's last barrier
        __syncwarp();
        // the stage's scalars are read before the tile's first barrier: thread 0
        // refills this stage's slots when it starts tile j + 1, which it can do
        // once every thread has passed the tile's last barrier
        const int64_t E0 = sm.E0[st], E1 = sm.E1[st];
        const int64_t tg = AGG ? sm.tg[st] : 0;
        const float *Tg = sm.T[st] + sm.toff[st];   // group totals (grouping)
        const int64_t base = window_base(E0);
        const int64_t my0 = base + (int64_t)tid * KT;
        // window-relative (32-bit): the tile is [e0, e1), my positions [p0, p0 + KT)
        const int p0 = tid * KT, e0 = (int)(E0 - base), e1 = (int)(E1 - base);
        const uint32_t vmask = valid_mask32<KT>(e0 - p0, e1 - p0);
        constexpr uint32_t bmask = KT == 32 ? 0xffffffffu : ((1u << KT) - 1u);
        // ray starts among my edges, and ends: an edge ends a ray when the next
        // edge starts one or it is the tile's last edge (positions outside the
        // tile are neutral, so their bits do not matter)
        // the bitmap words covering my edges (a thread's KT bits start at a
        // multiple of 8 within a word, so with KT > 8 they can straddle two)
        constexpr bool kEnds2 = KT > 8;
        const int wi = (int)(((base + p0) >> 5) - ((base >> 5) & ~(int64_t)3));
        const uint32_t hw0 = sm.hb[st][wi], hw1 = sm.hb[st][wi + 1];
        const uint32_t ew0 = AGG ? sm.eb[st][AGG ? wi : 0] : 0u;
        const uint32_t ew1 = AGG && kEnds2 ? sm.eb[st][AGG ? wi + 1 : 0] : 0u;
        const uint32_t sh = ((uint32_t)base + (uint32_t)p0) & 31u;
        const uint64_t words = ((uint64_t)hw1 << 32) | hw0;
        const uint64_t bits = words >> sh;
        const uint32_t hbits = (uint32_t)bits & bmask;
        uint32_t tbits = (uint32_t)(bits >> 1) & bmask;
        const int last = e1 - 1 - p0;
        if ((unsigned)last < (unsigned)KT) tbits |= 1u << (uint32_t)last;

        // cavities (first pass: the initial message), nu
        float2 L[KP], nv[KP];
#pragma unroll
        for (int k = 0; k < KT; k += 4) {
            const float4 n4 = *reinterpret_cast<const float4 *>(&sm.nu[st][tid * KT + k]);
            nv[k / 2] = make_float2(n4.x, n4.y);
            nv[k / 2 + 1] = make_float2(n4.z, n4.w);
        }
        if (first) {
#pragma unroll
            for (int i = 0; i < KP; ++i) L[i] = splat(L0);
        } else {
#pragma unroll
            for (int k = 0; k < KT; k += 4) {
                float4 l4;
                if constexpr (is_bf16<LamT>()) {   // bf16 -> FP32 is exact: the bits move up
                    const uint2 u = *reinterpret_cast<const uint2 *>(&sm.lam[st][tid * KT + k]);
                    l4 = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
                } else {
                    l4 = *reinterpret_cast<const float4 *>(&sm.lam[st][tid * KT + k]);
                }
                float4 g4;
                if constexpr (AGG) {   // the total of each edge's group
                    const uint2 gg = *reinterpret_cast<const uint2 *>(&sm.gid[st][tid * KT + k]);
                    g4 = make_float4(Tg[gg.x & 0xffffu], Tg[gg.x >> 16], Tg[gg.y & 0xffffu], Tg[gg.y >> 16]);
                } else {
                    g4 = *reinterpret_cast<const float4 *>(&sm.T[st][tid * KT + k]);
                }
                L[k / 2] = add2(make_float2(g4.x, g4.y), make_float2(-l4.x, -l4.y));
                L[k / 2 + 1] = add2(make_float2(g4.z, g4.w), make_float2(-l4.z, -l4.w));
            }
        }
        if (vmask != bmask) {   // the threads at the tile's ends: positions outside it are neutral
#pragma unroll
            for (int k = 0; k < KT; ++k)
                if (!((vmask >> k) & 1u)) {
                    if (k & 1) L[k / 2].y = -INFINITY;
                    else L[k / 2].x = -INFINITY;
                }
        }
        float2 al[KP] = {}, be[KP] = {}, cc[KP] = {};   // set below (both forms), read through the lambdas
        auto AL = [&](int k) { return (k & 1) ? al[k / 2].y : al[k / 2].x; };
        auto BE = [&](int k) { return (k & 1) ? be[k / 2].y : be[k / 2].x; };
        auto CC = [&](int k) { return (k & 1) ? cc[k / 2].y : cc[k / 2].x; };
        auto put = [](float2 *a, int k, float v) {
            if (k & 1) a[k / 2].y = v;
            else a[k / 2].x = v;
        };
        // odds form (floored kernels): the forward and backward maps in front of
        // every edge, R_k = a_k + b_k R_in and beta_k = u_k + v_k beta_in
        float2 Ap[KP], Bp[KP], Up[KP], Vp[KP];
        float2 fagg, bagg;
        if constexpr (FL) {
            float2 tt[KP];
#pragma unroll
            for (int i = 0; i < KP; ++i) coeff_odds(L[i], nv[i], nu_ref, tt[i], al[i], be[i], cc[i]);
            // backward maps beta -> u + v beta (v = 0 from a ray end on), kept
            // in front of every edge (the state after it)
            Bwd ba = {0.f, 1.f};
#pragma unroll
            for (int k = KT - 1; k >= 0; --k) {
                if ((tbits >> k) & 1u) ba = {bg_x, 0.f};
                put(Up, k, ba.u);
                put(Vp, k, ba.v);
                ba.u = tile::step_B(ba.u, AL(k), BE(k), CC(k));
                ba.v = tile::step_P(ba.v, AL(k), BE(k));
            }
            // forward maps R -> a + b R (reset to the constant c at a ray
            // start), kept in front of every edge (the state before it)
            float fa_a = 0.f, fa_b = 1.f;
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if ((hbits >> k) & 1u) {
                    fa_a = nu_ref;
                    fa_b = 0.f;
                }
                put(Ap, k, fa_a);
                put(Bp, k, fa_b);
                const float tk = (k & 1) ? tt[k / 2].y : tt[k / 2].x;
                const float nk = (k & 1) ? nv[k / 2].y : nv[k / 2].x;
                fa_a = fmaf(tk, fa_a + nk, fa_a);
                fa_b = fmaf(tk, fa_b, fa_b);
            }
            fagg = make_float2(fminf(fa_a, kRmax), fminf(fa_b, kRmax));
            bagg = make_float2(ba.u, ba.v);
        } else {
#pragma unroll
            for (int i = 0; i < KP; ++i) coeff_pair(L[i], nv[i], nu_ref, al[i], be[i], cc[i]);
            // thread aggregates: forward map (A, P) -> (A + x P, y P) with the sign
            // of y marking a ray start; backward map B -> u + v B (v = 0 after a ray end)
            Fwd fa = {0.f, 1.f};
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if ((hbits >> k) & 1u) fa = {0.f, -1.f};
                fa.x = fmaf(fabsf(fa.y), CC(k), fa.x);
                fa.y = tile::step_P(fa.y, AL(k), BE(k));
            }
            Bwd ba = {0.f, 1.f};
#pragma unroll
            for (int k = KT - 1; k >= 0; --k) {
                if ((tbits >> k) & 1u) ba = {bg_x, 0.f};
                ba.u = tile::step_B(ba.u, AL(k), BE(k), CC(k));
                ba.v = tile::step_P(ba.v, AL(k), BE(k));
            }
            fagg = make_float2(fa.x, fa.y);
            bagg = make_float2(ba.u, ba.v);
        }
        constexpr int NA = S::NA;
        sm.fagg[agg_slot<NA, NT>(tid)] = fagg;
        sm.bagg[agg_slot<NA, NT>(tid)] = bagg;
        // half-way: the next tile's copy has had this tile's time so far to land
        const bool ok = j + 1 < n ? mbar_wait(&sm.bar[(j + 1) & 1], ((j + 1) >> 1) & 1) : true;
        if (__syncthreads_or(!ok)) {   // also publishes the aggregates
            if (tid == 0) atomicOr(err, 2u);
            // drain this thread's own cp.async copies (the next tile's group
            // keys) before the CTA's shared memory is released.  A bulk copy
            // that never completed is abandoned with the CTA; the error word
            // tells the host, which must not use the context's results (the
            // context reports MRF_ETIMEOUT and must be reset).
            cp_async_wait<0>();
            return;
        }
        // warps 0 and 1 scan, the others gather the next tile meanwhile (then
        // warps 0 and 1 gather their share)
        if (tid < 32) {
            if constexpr (FL) scan_fwd_warp_odds<NT, NA>(sm.fagg);
            else scan_fwd_warp<NT, NA>(sm.fagg);
        } else if (tid < 64) {
            scan_bwd_warp<NT, NA>(sm.bagg);
        }
        if (j + 1 < n) gather(j + 1);
        __syncthreads();
        const float2 fi = sm.fagg[agg_slot<NA, NT>(tid)];
        const float2 bi = sm.bagg[agg_slot<NA, NT>(tid)];

        if constexpr (FL) {
            // the states at the thread's first edge, then every edge's R and
            // beta from the maps in front of it, and the messages, into nv[]
            const float Rin = fminf(fmaf(fi.y, nu_ref, fi.x), kRmax);
            const float Bin = fmaf(bi.y, bg_x, bi.x);
#pragma unroll
            for (int i = 0; i < KP; ++i) {
                const float2 R = fma2(Bp[i], splat(Rin), Ap[i]);
                const float2 beta = fma2(Vp[i], splat(Bin), Up[i]);
                nv[i] = message_pair_odds(R, nv[i], beta);
            }
        } else {
            // beta_i (exclusive suffix state) for every edge, into L[]
            {
                float B = fmaf(bi.y, bg_x, bi.x);
#pragma unroll
                for (int k = KT - 1; k >= 0; --k) {
                    if ((tbits >> k) & 1u) B = bg_x;
                    put(L, k, B);
                    B = tile::step_B(B, AL(k), BE(k), CC(k));
                }
            }
            // forward pass and the messages, two edges at a time, into nv[]
            {
                float X = fi.x, Y = fabsf(fi.y);
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    float2 Xp, Yp;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = 2 * i + h;
                        if ((hbits >> k) & 1u) {
                            X = 0.f;
                            Y = 1.f;
                        }
                        if (h) {
                            Xp.y = X;
                            Yp.y = Y;
                        } else {
                            Xp.x = X;
                            Yp.x = Y;
                        }
                        X = fmaf(Y, CC(k), X);
                        Y = tile::step_P(Y, AL(k), BE(k));
                    }
                    nv[i] = make_float2(tile::message<false>(Xp.x, Yp.x, nv[i].x, L[i].x, nu_ref),
                                        tile::message<false>(Xp.y, Yp.y, nv[i].y, L[i].y, nu_ref));
                }
            }
        }
        float lamv[KT];
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            lamv[2 * i] = nv[i].x;
            lamv[2 * i + 1] = nv[i].y;
        }
        if constexpr (is_bf16<LamT>()) {
            // store the rounded messages; the voxel totals below sum the same
            // rounded values, so the next cavity removes exactly what was added
            uint32_t hb16[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                hb16[k] = __bfloat16_as_ushort(__float2bfloat16_rn(lamv[k]));
                lamv[k] = __uint_as_float(hb16[k] << 16);
            }
            if (vmask == bmask) {
#pragma unroll
                for (int k = 0; k < KT; k += 4)
                    *reinterpret_cast<uint2 *>(lam + my0 + k) =
                        make_uint2(hb16[k] | (hb16[k + 1] << 16), hb16[k + 2] | (hb16[k + 3] << 16));
            } else {
#pragma unroll
                for (int k = 0; k < KT; ++k)
                    if ((vmask >> k) & 1u) lam[my0 + k] = __ushort_as_bfloat16((unsigned short)hb16[k]);
            }
        } else {
            if (vmask == bmask) {
#pragma unroll
                for (int k = 0; k < KT; k += 4)
                    *reinterpret_cast<float4 *>(lam + my0 + k) =
                        make_float4(lamv[k], lamv[k + 1], lamv[k + 2], lamv[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < KT; ++k)
                    if ((vmask >> k) & 1u) lam[my0 + k] = lamv[k];
            }
        }
        if (AGG) {
            // One partial sum per (tile, voxel) group.  The tile's messages go to
            // shared memory by window index (over the gathered T values, no longer
            // needed); position q of the tile's voxel order reads its message
            // through lx.  Group g of the tile (in voxel order) lands in slot
            // tg + g, and a position's window entry in gid is its group, so the
            // group that ends first among a thread's positions is the group of
            // its first position (group 0 if that lies before the tile).  In one
            // pass over its positions a thread stores the sums of the groups
            // that begin and end with it, keeps the head of its first group and
            // publishes what follows its last group end (all of it if it has
            // none); after the barrier the thread holding a group's end adds the
            // tails of the earlier threads back to the one where the group began.
            // Positions outside the tile belong to the first thread (before E0:
            // masked to 0) or come after the tile's last group end (never summed
            // into a partial).
            float *sl = sm.nu[st];
#pragma unroll
            for (int k = 0; k < KT; k += 4)
                *reinterpret_cast<float4 *>(&sl[tid * KT + k]) = make_float4(lamv[k], lamv[k + 1], lamv[k + 2], lamv[k + 3]);
            const uint32_t ebits =
                (uint32_t)((((uint64_t)ew1 << 32) | ew0) >> sh) & bmask & vmask;
            const uint32_t efirst = ebits & (0u - ebits);   // the thread's first group end
            const uint32_t erest = ebits ^ efirst;
            __syncthreads();
            const uint16_t *lxs = sm.lx[st];
            float x[KT];
            uint32_t w0 = 0;
#pragma unroll
            for (int k = 0; k < KT; k += 4) {
                const uint2 w2 = *reinterpret_cast<const uint2 *>(&lxs[tid * KT + k]);
                if (k == 0) w0 = w2.x & 0xffffu;
                x[k] = sl[w2.x & 0xffffu];
                x[k + 1] = sl[w2.x >> 16];
                x[k + 2] = sl[w2.y & 0xffffu];
                x[k + 3] = sl[w2.y >> 16];
            }
            // a thread whose first position lies before the tile's first edge
            // (E0 - base < 8) ends group 0 first, if it ends any
            const uint32_t g0 = p0 > e0 ? (uint32_t)sm.gid[st][w0] : 0u;
            if (vmask != bmask) {
#pragma unroll
                for (int k = 0; k < KT; ++k)
                    if (!((vmask >> k) & 1u)) x[k] = 0.f;
            }
            float *out = partial + tg + g0;
            float acc = 0.f, head = 0.f;
            int r = 0;
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                acc += x[k];
                if ((efirst >> k) & 1u) {
                    head = acc;
                    acc = 0.f;
                }
                if ((erest >> k) & 1u) {
                    out[++r] = acc;
                    acc = 0.f;
                }
            }
            float2 *tails = sm.tail;
            tails[tid] = make_float2(acc, ebits ? 1.f : 0.f);
            cp_async_wait<0>();   // the next tile's gathers: in for every thread after the barrier below
            __syncthreads();      // the tails are in
            if (ebits) {
                float carry = 0.f;
                for (int t = tid - 1; t >= 0; --t) {
                    const float2 e = tails[t];
                    carry += e.x;
                    if (e.y != 0.f) break;
                }
                out[0] = carry + head;
            }
        }
        // with grouping, the epilogue's barriers come after every read of this
        // stage's scan results; without it, one barrier keeps thread 0 from
        // refilling the stage before the slowest thread has read them
        if (!AGG) __syncthreads();
    }
}

// The failure path of the bounded waits, exercised on purpose: one CTA waits
// on an mbarrier that nothing arrives on, gives up after the time limit, and
// reports it through the error word as the ray kernel does.
__global__ void k_wait_probe(uint32_t *__restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, 4u);
}

// Whole rays packed greedily into tiles of at most cap edges, counted from the
// tile's first edge rounded down to 8.  The packing restarts every
// kPackRays rays, so that chunks pack independently (a thread each) and only
// a chunk's last tile may be short.  Rays without edges belong to no tile.
constexpr int64_t kPackRays = 512;

__device__ __forceinline__ int64_t pack_chunk(const int64_t *__restrict__ ro, int64_t r, int64_t rend, int64_t cap,
                                              int64_t *__restrict__ out) {
    int64_t n = 0;
    while (r < rend && ro[r + 1] == ro[r]) ++r;
    while (r < rend) {
        const int64_t base = ro[r] & ~(int64_t)7;
        if (out) out[n] = ro[r];
        ++n;
        int64_t q = r + 1;
        while (q < rend && ro[q + 1] - base <= cap) ++q;
        r = q;
    }
    return n;
}

// counts[c] = the tiles of chunk c; with tile_off, writes their first edges
__global__ void k_tile_pack(const int64_t *__restrict__ ray_off, int64_t R, int64_t cap, int32_t *__restrict__ counts,
                            const int64_t *__restrict__ tile_off, int64_t *__restrict__ tile_E) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = c * kPackRays;
    if (r0 >= R) return;
    const int64_t r1 = r0 + kPackRays < R ? r0 + kPackRays : R;
    if (tile_off) pack_chunk(ray_off, r0, r1, cap, tile_E + tile_off[c]);
    else counts[c] = (int32_t)pack_chunk(ray_off, r0, r1, cap, nullptr);
}

// tile_E[t] = ray_off[tile_r0[t]]
__global__ void k_tile_edges(const int64_t *__restrict__ ray_off, const uint32_t *__restrict__ tile_r0,
                             int64_t ntiles, int64_t *__restrict__ tile_E) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= ntiles) tile_E[t] = ray_off[tile_r0[t]];
}

// bit e of hb set iff edge e is the first edge of a ray
__global__ void k_ray_starts(const int64_t *__restrict__ ray_off, int64_t R, uint32_t *__restrict__ hb) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t a = ray_off[r];
    if (ray_off[r + 1] > a) atomicOr(&hb[a >> 5], 1u << (uint32_t)(a & 31));
}

__global__ void k_bf16_to_f32(const uint16_t *__restrict__ in, float *__restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __uint_as_float((uint32_t)in[i] << 16);
}

template <int KT, bool AGG, int NT, typename LamT, bool FL = false>
cudaError_t launch_pipe(int64_t grid, const int64_t *tile_E, int64_t ntiles, const uint32_t *hb, const uint32_t *vox,
                        const float *nu, const float *T, void *lam, float nu_bg, float nu_ref, int first, float L0, uint32_t *err,
                        const uint16_t *lidx, const uint32_t *ends, const uint16_t *gid, const uint32_t *gkey,
                        const int64_t *tg_off, float *partial,
                        cudaStream_t s) {
    static int per_sm = 0;   // resident CTAs per SM, from the occupancy calculator
    const int bytes = (int)sizeof(PipeSmem<KT, NT, LamT, AGG>);
    if (per_sm == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(k_ray_pipe<KT, AGG, NT, LamT, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ray_pipe<KT, AGG, NT, LamT, FL>, NT, bytes);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    }
    grid *= per_sm;   // callers pass the SM count
    if (grid > ntiles) grid = ntiles;
    k_ray_pipe<KT, AGG, NT, LamT, FL><<<(unsigned)grid, NT, bytes, s>>>(
        tile_E, ntiles, hb, vox, nu, T, static_cast<LamT *>(lam), nu_bg, nu_ref, first, L0, err, lidx, ends, gid, gkey, tg_off,
        partial);
    return cudaGetLastError();
}

}  // namespace

bool ray_pipe_supported(int kt, int nt) {
    return (nt == kThreads && (kt == 8 || kt == 16)) || (nt == 128 && kt == 16) || (nt == 512 && kt == 4);
}

int64_t tile_pack_chunks(int64_t R) { return ceil_div(R, kPackRays); }

cudaError_t launch_tile_pack(const int64_t *ray_off, int64_t R, int64_t cap, int32_t *counts, const int64_t *tile_off,
                             int64_t *tile_E, cudaStream_t s) {
    const int64_t nc = tile_pack_chunks(R);
    if (nc <= 0) return cudaSuccess;
    k_tile_pack<<<(unsigned)ceil_div(nc, 128), 128, 0, s>>>(ray_off, R, cap, counts, tile_off, tile_E);
    return cudaGetLastError();
}

cudaError_t launch_ray_pipe_plan(const int64_t *ray_off, int64_t R, const uint32_t *tile_r0, int64_t ntiles,
                                 int64_t *tile_E, uint32_t *hb, int64_t hb_words, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hb, 0, (size_t)hb_words * 4, s);
    if (e != cudaSuccess) return e;
    if (tile_E && tile_r0 && ntiles > 0)
        k_tile_edges<<<(unsigned)ceil_div(ntiles + 1, kThreads), kThreads, 0, s>>>(ray_off, tile_r0, ntiles, tile_E);
    if (R > 0) k_ray_starts<<<(unsigned)ceil_div(R, kThreads), kThreads, 0, s>>>(ray_off, R, hb);
    return cudaGetLastError();
}

cudaError_t launch_ray_pipe(int kt, int nt, bool bf16, int64_t n_sm, const int64_t *tile_E, int64_t ntiles,
                            const uint32_t *hb, const uint32_t *vox, const float *nu, const float *T, void *lam,
                            float nu_bg, float nu_ref, int first, float L0, uint32_t *err, const uint16_t *lidx,
                            const uint32_t *ends, const uint16_t *gid, const uint32_t *gkey, const int64_t *tg_off,
                            float *partial, cudaStream_t s, bool floored) {
    if (ntiles <= 0) return cudaSuccess;
    const bool agg = partial != nullptr;
    if (bf16 && !agg) return cudaErrorInvalidValue;   // bf16 storage is for the grouped path only
#define MRF_PIPE(KT, AGG, NT, LT)                                                                                   \
    return launch_pipe<KT, AGG, NT, LT>(n_sm, tile_E, ntiles, hb, vox, nu, T, lam, nu_bg, nu_ref, first, L0, err,   \
                                        lidx, ends, gid, gkey, tg_off, partial, s)
#define MRF_PIPE_FL(KT, AGG, NT, LT)                                                                                \
    return launch_pipe<KT, AGG, NT, LT, true>(n_sm, tile_E, ntiles, hb, vox, nu, T, lam, nu_bg, nu_ref, first, L0,  \
                                              err, lidx, ends, gid, gkey, tg_off, partial, s)
    // the grouped 256-thread shapes also come in the floored form (message())
    if (nt == kThreads && kt == 8) {
        if (bf16 && floored) MRF_PIPE_FL(8, true, kThreads, __nv_bfloat16);
        if (bf16) MRF_PIPE(8, true, kThreads, __nv_bfloat16);
        if (agg && floored) MRF_PIPE_FL(8, true, kThreads, float);
        if (agg) MRF_PIPE(8, true, kThreads, float);
        MRF_PIPE(8, false, kThreads, float);
    }
    if (nt == kThreads && kt == 16) {
        if (bf16 && floored) MRF_PIPE_FL(16, true, kThreads, __nv_bfloat16);
        if (bf16) MRF_PIPE(16, true, kThreads, __nv_bfloat16);
        if (agg && floored) MRF_PIPE_FL(16, true, kThreads, float);
        if (agg) MRF_PIPE(16, true, kThreads, float);
        MRF_PIPE(16, false, kThreads, float);
    }
    if (nt == 128 && kt == 16) {
        if (bf16) MRF_PIPE(16, true, 128, __nv_bfloat16);
        if (agg) MRF_PIPE(16, true, 128, float);
        MRF_PIPE(16, false, 128, float);
    }
    if (nt == 512 && kt == 4) {
        if (bf16) MRF_PIPE(4, true, 512, __nv_bfloat16);
        if (agg) MRF_PIPE(4, true, 512, float);
        MRF_PIPE(4, false, 512, float);
    }
#undef MRF_PIPE
#undef MRF_PIPE_FL
    return cudaErrorInvalidValue;
}

cudaError_t launch_wait_probe(uint32_t *err, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t launch_bf16_to_f32(const void *in, float *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_bf16_to_f32<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(static_cast<const uint16_t *>(in), out, n);
    return cudaGetLastError();
}

}  // namespace mrf
