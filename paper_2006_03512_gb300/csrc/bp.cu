// Loopy-BP kernels on caller buffers and the voxel totals: the standalone
// ray -> voxel message kernel (Eqs. "pos"/"neg"; the arithmetic is in
// ray_tile.cuh), the voxel totals (the marginal equation; cavities of Eq.
// "node_to_factor"), the plain FP64 form, plans and small helpers.
#include <math.h>

#include "mrf_internal.cuh"
#include "ray_tile.cuh"
#include "seg_scan.cuh"


namespace mrf {
namespace {

using tile::Bwd;
using tile::Fwd;

// ------------------------------------------------- ray -> voxel, standalone
// One CTA per tile of whole rays, read straight from global memory (no
// padding is assumed after the caller's arrays).
template <int KT>
__global__ void __launch_bounds__(kThreads, KT == 8 ? 3 : 2)
    k_ray_messages(const int64_t *__restrict__ ray_off, const uint32_t *__restrict__ tile_r0,
                   const uint32_t *__restrict__ vox, const float *__restrict__ nu, const float *__restrict__ T,
                   float *__restrict__ lam, int64_t n_alloc, float nu_bg, float nu_ref, int first, float L0,
                   int aligned, uint32_t *__restrict__ err, const float *__restrict__ wlen) {
    constexpr int CAP = kThreads * KT;
    constexpr int NW = CAP / 32;
    __shared__ uint32_t s_head[NW], s_tail[NW];
    __shared__ Fwd s_fw[2 * kThreads / 32];
    __shared__ Bwd s_bw[2 * kThreads / 32];

    const uint32_t ra = tile_r0[blockIdx.x], rb = tile_r0[blockIdx.x + 1];
    if (ra >= rb) return;
    const int64_t E0 = ray_off[ra], E1 = ray_off[rb];
    if (E1 <= E0) return;
    const int64_t base = E0 & ~(int64_t)3;
    if (E1 - base > CAP) {  // only if the caller's longest-ray bound was too small
        if (threadIdx.x == 0 && err) atomicOr(err, 1u);
        return;
    }
    for (int i = threadIdx.x; i < NW; i += kThreads) {
        s_head[i] = 0u;
        s_tail[i] = 0u;
    }
    __syncthreads();
    for (uint32_t r = ra + threadIdx.x; r < rb; r += kThreads) {
        const int64_t a = ray_off[r], b = ray_off[r + 1];
        if (b > a) {
            const int ia = (int)(a - base), ib = (int)(b - 1 - base);
            atomicOr(&s_head[ia >> 5], 1u << (ia & 31));
            atomicOr(&s_tail[ib >> 5], 1u << (ib & 31));
        }
    }
    __syncthreads();

    const int64_t my0 = base + (int64_t)threadIdx.x * KT;
    const int bit0 = threadIdx.x * KT;
    const uint32_t bmask = KT == 32 ? 0xffffffffu : ((1u << KT) - 1u);
    const uint32_t hbits = (s_head[bit0 >> 5] >> (bit0 & 31)) & bmask;
    const uint32_t tbits = (s_tail[bit0 >> 5] >> (bit0 & 31)) & bmask;
    const uint32_t vmask = tile::valid_mask<KT>(my0, E0, E1);

    float nv[KT], lo[KT];
    uint32_t vx[KT];
    if (aligned && my0 + KT <= n_alloc) {
#pragma unroll
        for (int k = 0; k < KT; k += 4) {
            const float4 n4 = __ldg(reinterpret_cast<const float4 *>(nu + my0 + k));
            nv[k] = n4.x; nv[k + 1] = n4.y; nv[k + 2] = n4.z; nv[k + 3] = n4.w;
            if (!first) {
                const uint4 v4 = __ldg(reinterpret_cast<const uint4 *>(vox + my0 + k));
                vx[k] = v4.x; vx[k + 1] = v4.y; vx[k + 2] = v4.z; vx[k + 3] = v4.w;
                const float4 l4 = *reinterpret_cast<const float4 *>(lam + my0 + k);
                lo[k] = l4.x; lo[k + 1] = l4.y; lo[k + 2] = l4.z; lo[k + 3] = l4.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const bool in = (vmask >> k) & 1u;
            nv[k] = in ? nu[my0 + k] : 0.f;
            if (!first) {
                vx[k] = in ? vox[my0 + k] : 0u;
                lo[k] = in ? lam[my0 + k] : 0.f;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const bool in = (vmask >> k) & 1u;
        lo[k] = first ? L0 : (in ? __ldg(T + vx[k]) - lo[k] : 0.f);
    }
    tile::tile_messages<KT>(nv, lo, vmask, hbits, tbits, nu_bg, nu_ref, s_fw, s_bw);
    if (wlen) {   // traversed-length weighting: what is stored (and summed) is w lambda
#pragma unroll
        for (int k = 0; k < KT; ++k)
            if ((vmask >> k) & 1u) nv[k] *= __ldg(wlen + my0 + k);
    }
    if (vmask == bmask && aligned) {
#pragma unroll
        for (int k = 0; k < KT; k += 4)
            *reinterpret_cast<float4 *>(lam + my0 + k) = make_float4(nv[k], nv[k + 1], nv[k + 2], nv[k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < KT; ++k)
            if ((vmask >> k) & 1u) lam[my0 + k] = nv[k];
    }
}

// ------------------------------------------------- long rays in FP64
// The messages of the rays listed in ids (one thread each), from the FP32
// context's own cavities (L = T[v] - lambda_old, or L0 in the first pass) and
// FP32 likelihoods, with the prefix and suffix recurrences (Eqs. "pos" /
// "neg" as A, P, B: the plain FP64 form) accumulated in FP64; written, as FP32,
// to out[loff[j] ...] (the FP32 ray kernel overwrites lam afterwards; the
// scatter below puts these back).  bscr: FP64 scratch of the same layout.
__global__ void k_long_rays_f64(const int64_t *__restrict__ ray_off, const uint32_t *__restrict__ ids,
                                int64_t n_long, const int64_t *__restrict__ loff, const uint32_t *__restrict__ vox,
                                const float *__restrict__ nu, const float *__restrict__ T,
                                const float *__restrict__ lam, int first, double L0, double nu_bg,
                                float *__restrict__ out, double *__restrict__ bscr) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_long) return;
    const int64_t e0 = ray_off[ids[j]], e1 = ray_off[ids[j] + 1], o = loff[j];
    auto cavity = [&](int64_t e) -> double { return first ? L0 : (double)(T[vox[e]] - lam[e]); };
    double B = nu_bg;
    for (int64_t e = e1 - 1; e >= e0; --e) {
        const double L = cavity(e);
        const double ex = exp(-fabs(L));
        const double rr = 1.0 / (1.0 + ex);
        const double m1 = L >= 0.0 ? rr : ex * rr;
        const double m0 = L >= 0.0 ? ex * rr : rr;
        bscr[o + (e - e0)] = B;
        B = m1 * (double)nu[e] + m0 * B;
    }
    double X = 0.0, Y = 1.0;
    for (int64_t e = e0; e < e1; ++e) {
        const double L = cavity(e);
        const double ex = exp(-fabs(L));
        const double rr = 1.0 / (1.0 + ex);
        const double m1 = L >= 0.0 ? rr : ex * rr;
        const double m0 = L >= 0.0 ? ex * rr : rr;
        const double n = (double)nu[e];
        double l = log(X + Y * n) - log(X + Y * bscr[o + (e - e0)]);
        if (l != l) l = 0.0;
        l = l > 64.0 ? 64.0 : (l < -64.0 ? -64.0 : l);
        out[o + (e - e0)] = (float)l;
        X = X + Y * m1 * n;
        Y = Y * m0;
    }
}

// lam[edges of long ray j] = out[loff[j] ...]
__global__ void k_long_scatter(const int64_t *__restrict__ ray_off, const uint32_t *__restrict__ ids,
                               int64_t n_long, const int64_t *__restrict__ loff, const float *__restrict__ out,
                               float *__restrict__ lam) {
    const int64_t j = (int64_t)blockIdx.x;   // one warp per long ray
    if (j >= n_long) return;
    const int64_t e0 = ray_off[ids[j]], n = ray_off[ids[j] + 1] - e0, o = loff[j];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) lam[e0 + i] = out[o + i];
}

// tile_r0[t] = first ray r with ray_off[r] >= min(t * window, E)
__global__ void k_ray_plan(const int64_t *__restrict__ ray_off, int64_t R, int64_t E, int64_t window,
                           uint32_t *__restrict__ tile_r0, int64_t ntiles) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    int64_t x = t * window;
    if (x > E) x = E;
    int64_t lo = 0, hi = R;  // answer in [0, R]; ray_off[R] = E >= x
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ray_off[mid] >= x) hi = mid;
        else lo = mid + 1;
    }
    tile_r0[t] = (uint32_t)lo;
}

// ----------------------------------------------------- voxel totals (FP32/64)
using seg::SegAgg;
using seg::acc_add;
using seg::block_seg_exclusive;
using seg::seg_op;

// plan[2t] = segment containing position t*kTile, plan[2t+1] = segment containing
// the tile's last position.
__global__ void k_reduce_plan(const uint32_t *__restrict__ seg_off, int64_t S, int64_t E,
                              uint32_t *__restrict__ plan, int64_t ntiles) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int64_t p0 = t * kTile;
    const int64_t p1 = (p0 + kTile < E ? p0 + kTile : E) - 1;
    for (int j = 0; j < 2; ++j) {
        const int64_t x = j ? p1 : p0;
        int64_t lo = 0, hi = S - 1;  // last s with seg_off[s] <= x
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if ((int64_t)seg_off[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        plan[2 * t + j] = (uint32_t)lo;
    }
}

// FP32: five CTAs per SM (48 registers, no spills) keep more gathers in flight
template <typename V, bool KAHAN>
__global__ void __launch_bounds__(kThreads, sizeof(V) == 4 ? 5 : 1)
    k_voxel_reduce(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ seg_off,
                   const uint32_t *__restrict__ seg_vox, const uint32_t *__restrict__ plan,
                   const V *__restrict__ lam, V *__restrict__ T, V logit_prior, int64_t E, int64_t n_alloc,
                   V *__restrict__ head_part, V *__restrict__ tail_part, uint32_t *__restrict__ tail_seg,
                   int aligned) {
    __shared__ uint32_t s_end[kTile / 32];
    __shared__ SegAgg<V> s_w[kThreads / 32];
    __shared__ int s_cont;
    const int64_t P0 = (int64_t)blockIdx.x * kTile;
    const int64_t P1 = P0 + kTile < E ? P0 + kTile : E;
    // this thread's values first: their index loads and gathers are in flight
    // while the segment ends are marked below
    const int64_t q0 = P0 + (int64_t)threadIdx.x * kItems;
    V x[kItems];
    if (aligned && q0 + kItems <= n_alloc && q0 + kItems <= P1) {
        uint32_t pm[kItems];
#pragma unroll
        for (int k = 0; k < kItems; k += 4) {
            const uint4 p4 = __ldg(reinterpret_cast<const uint4 *>(perm + q0 + k));
            pm[k] = p4.x; pm[k + 1] = p4.y; pm[k + 2] = p4.z; pm[k + 3] = p4.w;
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) x[k] = __ldg(lam + pm[k]);
    } else {
#pragma unroll
        for (int k = 0; k < kItems; ++k) x[k] = (q0 + k < P1) ? __ldg(lam + perm[q0 + k]) : (V)0;
    }
    const uint32_t s_lo = plan[2 * blockIdx.x], s_hi = plan[2 * blockIdx.x + 1];
    for (int i = threadIdx.x; i < kTile / 32; i += kThreads) s_end[i] = 0u;
    if (threadIdx.x == 0) s_cont = (int64_t)seg_off[s_lo] < P0;
    __syncthreads();
    for (int64_t s = (int64_t)s_lo + threadIdx.x; s <= (int64_t)s_hi; s += kThreads) {
        const int64_t endp = (int64_t)seg_off[s + 1] - 1;
        if (endp >= P0 && endp < P1) {
            const int b = (int)(endp - P0);
            atomicOr(&s_end[b >> 5], 1u << (b & 31));
        }
    }
    __syncthreads();
    const int bit0 = threadIdx.x * kItems;
    const uint32_t ebits = (s_end[bit0 >> 5] >> (bit0 & 31)) & ((1u << kItems) - 1u);
    // thread aggregate: sum after the last end in this thread, number of ends
    SegAgg<V> agg = {(V)0, (V)0, 0};
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        acc_add<KAHAN>(agg.s, agg.cs, x[k]);
        if ((ebits >> k) & 1u) {
            agg.n += 1;
            agg.s = (V)0;
            agg.cs = (V)0;
        }
    }
    const SegAgg<V> carry = block_seg_exclusive(agg, s_w);
    // emit every segment that ends in this thread
    V s = (V)0, cs = (V)0;
    int nend = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        acc_add<KAHAN>(s, cs, x[k]);
        if ((ebits >> k) & 1u) {
            V total = s - cs;
            if (nend == 0) total = (carry.s - carry.cs) + total;
            const uint32_t seg = s_lo + (uint32_t)(carry.n + nend);
            if (seg == s_lo && s_cont) head_part[blockIdx.x] = total;
            else T[seg_vox[seg]] = logit_prior + total;
            ++nend;
            s = (V)0;
            cs = (V)0;
        }
    }
    // the thread holding the tile's last position records the open segment
    if (q0 <= P1 - 1 && P1 - 1 < q0 + kItems) {
        const int klast = (int)(P1 - 1 - q0);
        if ((ebits >> klast) & 1u) {
            tail_seg[blockIdx.x] = kNone;
        } else {
            const V open = nend ? (s - cs) : (carry.s - carry.cs) + (s - cs);
            if (s_lo == s_hi && s_cont) {
                head_part[blockIdx.x] = open;
                tail_seg[blockIdx.x] = kNone;
            } else {
                tail_part[blockIdx.x] = open;
                tail_seg[blockIdx.x] = s_hi;
            }
        }
    }
}

// Segments that cross tile boundaries: the tile where a segment starts adds the
// partial sums of the following tiles, in tile order.
template <typename V>
__global__ void k_reduce_fixup(const uint32_t *__restrict__ seg_off, const uint32_t *__restrict__ seg_vox,
                               const V *__restrict__ head_part, const V *__restrict__ tail_part,
                               const uint32_t *__restrict__ tail_seg, V *__restrict__ T, V logit_prior,
                               int64_t ntiles) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t s = tail_seg[t];
    if (s == kNone) return;
    const int64_t end = seg_off[s + 1];
    V sum = tail_part[t];
    for (int64_t u = t + 1; u < ntiles; ++u) {
        sum += head_part[u];
        if (end <= (u + 1) * kTile) break;
    }
    T[seg_vox[s]] = logit_prior + sum;
}

// ---------------------------------------------------------- plain FP64 form
// One thread per ray, two sequential passes (backward for B, forward for A, P
// and the messages), FP64 throughout.  Comparator for the FP32 path.
__global__ void __launch_bounds__(kThreads)
    k_ray_messages_f64(const int64_t *__restrict__ ray_off, int64_t R, const uint32_t *__restrict__ vox,
                       const double *__restrict__ nu, const double *__restrict__ T, double *__restrict__ lam,
                       double *__restrict__ bscr, double nu_bg, int first, double L0) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = ray_off[r], e1 = ray_off[r + 1];
        if (e1 <= e0) continue;
        double B = nu_bg;
        for (int64_t e = e1 - 1; e >= e0; --e) {
            const double L = first ? L0 : T[vox[e]] - lam[e];
            const double ex = exp(-fabs(L));
            const double rr = 1.0 / (1.0 + ex);
            const double m1 = L >= 0.0 ? rr : ex * rr;
            const double m0 = L >= 0.0 ? ex * rr : rr;
            bscr[e] = B;
            B = m1 * nu[e] + m0 * B;
        }
        double X = 0.0, Y = 1.0;
        for (int64_t e = e0; e < e1; ++e) {
            const double L = first ? L0 : T[vox[e]] - lam[e];
            const double ex = exp(-fabs(L));
            const double rr = 1.0 / (1.0 + ex);
            const double m1 = L >= 0.0 ? rr : ex * rr;
            const double m0 = L >= 0.0 ? ex * rr : rr;
            const double num = X + Y * nu[e];
            const double den = X + Y * bscr[e];
            double l = log(num) - log(den);
            if (l != l) l = 0.0;
            l = l > 64.0 ? 64.0 : (l < -64.0 ? -64.0 : l);
            lam[e] = l;
            X = X + Y * m1 * nu[e];
            Y = Y * m0;
        }
    }
}

// --------------------------------------- log-domain FP32 form (an ablation)
// The messages of Eqs. "pos"/"neg" evaluated as the paper does, in the log
// domain, here in FP32: log P_i = sum_{k<i} log m0_k (Kahan-compensated),
// log A_i = log sum_{j<i} m1_j nu_j P_j and log B_i by log-add-exp
// recurrences, log pos_i = lae(log A_i, log P_i + log nu_i), log neg_i =
// lae(log A_i, log P_i + log B_i), lambda_i = log pos_i - log neg_i.  One thread
// per ray, two sequential passes, library logf/expf/log1pf.
__device__ __forceinline__ float log_add_exp(float a, float b) {
    const float m = fmaxf(a, b);
    if (m == -INFINITY) return -INFINITY;
    return m + log1pf(expf(-fabsf(a - b)));
}
__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

__global__ void __launch_bounds__(kThreads)
    k_ray_messages_log32(const int64_t *__restrict__ ray_off, int64_t R, const uint32_t *__restrict__ vox,
                         const float *__restrict__ nu, const float *__restrict__ T, float *__restrict__ lam,
                         float *__restrict__ lbscr, float nu_bg, int first, float L0) {
    const float lbg = logf(nu_bg);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = ray_off[r], e1 = ray_off[r + 1];
        if (e1 <= e0) continue;
        float lB = lbg;   // log B after the ray's last voxel
        for (int64_t e = e1 - 1; e >= e0; --e) {
            const float L = first ? L0 : T[vox[e]] - lam[e];
            lbscr[e] = lB;
            lB = log_add_exp(logf(nu[e]) - softplus(-L), lB - softplus(L));   // m1 nu + m0 B
        }
        float lA = -INFINITY, lP = 0.f, comp = 0.f;
        for (int64_t e = e0; e < e1; ++e) {
            const float L = first ? L0 : T[vox[e]] - lam[e];
            const float lnu = logf(nu[e]);
            const float lpos = log_add_exp(lA, lP + lnu);
            const float lneg = log_add_exp(lA, lP + lbscr[e]);
            float l = lpos - lneg;
            if (l != l) l = 0.f;
            lam[e] = fminf(fmaxf(l, -64.f), 64.f);
            lA = log_add_exp(lA, lnu - softplus(-L) + lP);
            const float y = -softplus(L) - comp;   // Kahan: lP += log m0
            const float t = lP + y;
            comp = (t - lP) - y;
            lP = t;
        }
    }
}

// ------------------------------------------------------------------ helpers
template <typename V>
__global__ void k_fill(V *__restrict__ p, int64_t n, V v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

template <typename V>
__global__ void k_marginals(const V *__restrict__ T, float *__restrict__ p, GridMap gm) {
    const int64_t n = (int64_t)gm.nx * gm.ny * gm.nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(i % gm.nx), y = (uint32_t)((i / gm.nx) % gm.ny), z = (uint32_t)(i / ((int64_t)gm.nx * gm.ny));
        const V t = T[voxel_key(x, y, z, gm.nbx, gm.nby)];
        p[i] = (float)((V)1 / ((V)1 + exp(-t)));
    }
}

template <typename V>
__global__ void k_gather_linear(const V *__restrict__ T, V *__restrict__ out, GridMap gm) {
    const int64_t n = (int64_t)gm.nx * gm.ny * gm.nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(i % gm.nx), y = (uint32_t)((i / gm.nx) % gm.ny), z = (uint32_t)(i / ((int64_t)gm.nx * gm.ny));
        out[i] = T[voxel_key(x, y, z, gm.nbx, gm.nby)];
    }
}

__global__ void k_keys_to_linear(const uint32_t *__restrict__ keys, uint32_t *__restrict__ out, int64_t n, GridMap gm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x, y, z;
        key_xyz(keys[i], gm.nbx, gm.nby, x, y, z);
        out[i] = x + gm.nx * (y + gm.ny * z);
    }
}

__global__ void k_f64_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

inline unsigned grid_for(int64_t n) {
    int64_t g = ceil_div(n, kThreads);
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g > 0 ? g : 1);
}

template <typename V, bool KAHAN>
cudaError_t voxel_reduce(const uint32_t *perm, const uint32_t *seg_off, const uint32_t *seg_vox,
                         const uint32_t *plan, int64_t ntiles, const V *lam, V *T, V logit_prior, int64_t E,
                         int64_t n_alloc, V *head_part, V *tail_part, uint32_t *tail_seg, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const int aligned = ((uintptr_t)perm & 15u) == 0;
    k_voxel_reduce<V, KAHAN><<<(unsigned)ntiles, kThreads, 0, s>>>(perm, seg_off, seg_vox, plan, lam, T, logit_prior,
                                                                   E, n_alloc, head_part, tail_part, tail_seg,
                                                                   aligned);
    k_reduce_fixup<V><<<(unsigned)ceil_div(ntiles, kThreads), kThreads, 0, s>>>(seg_off, seg_vox, head_part,
                                                                                tail_part, tail_seg, T,
                                                                                logit_prior, ntiles);
    return cudaGetLastError();
}

}  // namespace

// Items per thread for the ray kernel: the smallest of 8, 16, 32 whose window
// keeps at least half of the CTA's capacity for rays that start in it (with a
// longest ray of 703 voxels, 2048-edge tiles still fill to 93% and run 1.5x
// faster than 4096-edge ones).
int ray_tile_items(int32_t max_len) {
    for (int kt = 8; kt <= 32; kt *= 2)
        if ((int64_t)max_len + 3 <= (int64_t)kThreads * kt / 2) return kt;
    if ((int64_t)max_len + 3 + 256 <= (int64_t)kThreads * 32) return 32;
    return 0;
}

int64_t ray_tile_window(int kt, int32_t max_len) { return (int64_t)kThreads * kt - (int64_t)max_len - 3; }

cudaError_t launch_ray_plan(const int64_t *ray_off, int64_t R, int64_t E, int64_t window, uint32_t *tile_r0,
                            int64_t ntiles, cudaStream_t s) {
    k_ray_plan<<<(unsigned)ceil_div(ntiles + 1, kThreads), kThreads, 0, s>>>(ray_off, R, E, window, tile_r0, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_ray_messages_f32(int kt, const int64_t *ray_off, const uint32_t *tile_r0, int64_t ntiles,
                                    const uint32_t *vox, const float *nu, const float *T, float *lam,
                                    int64_t n_alloc, float nu_bg, float nu_ref, int first, float L0, uint32_t *err,
                                    cudaStream_t s, const float *wlen) {
    if (ntiles <= 0) return cudaSuccess;
    const int aligned = (((uintptr_t)vox | (uintptr_t)nu | (uintptr_t)lam) & 15u) == 0;
    switch (kt) {
        case 8:
            k_ray_messages<8><<<(unsigned)ntiles, kThreads, 0, s>>>(ray_off, tile_r0, vox, nu, T, lam, n_alloc, nu_bg, nu_ref,
                                                                    first, L0, aligned, err, wlen);
            break;
        case 16:
            k_ray_messages<16><<<(unsigned)ntiles, kThreads, 0, s>>>(ray_off, tile_r0, vox, nu, T, lam, n_alloc,
                                                                     nu_bg, nu_ref, first, L0, aligned, err, wlen);
            break;
        case 32:
            k_ray_messages<32><<<(unsigned)ntiles, kThreads, 0, s>>>(ray_off, tile_r0, vox, nu, T, lam, n_alloc,
                                                                     nu_bg, nu_ref, first, L0, aligned, err, wlen);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_plan(const uint32_t *seg_off, int64_t n_seg, int64_t E, uint32_t *plan, int64_t ntiles,
                               cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_reduce_plan<<<(unsigned)ceil_div(ntiles, kThreads), kThreads, 0, s>>>(seg_off, n_seg, E, plan, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_voxel_reduce_f32(const uint32_t *perm, const uint32_t *seg_off, const uint32_t *seg_vox,
                                    const uint32_t *plan, int64_t ntiles, const float *lam, float *T,
                                    float logit_prior, int64_t E, float *head_part, float *tail_part,
                                    uint32_t *tail_seg, cudaStream_t s) {
    return voxel_reduce<float, true>(perm, seg_off, seg_vox, plan, ntiles, lam, T, logit_prior, E, E, head_part,
                                     tail_part, tail_seg, s);
}

cudaError_t launch_voxel_reduce_f64(const uint32_t *perm, const uint32_t *seg_off, const uint32_t *seg_vox,
                                    const uint32_t *plan, int64_t ntiles, const double *lam, double *T,
                                    double logit_prior, int64_t E, double *head_part, double *tail_part,
                                    uint32_t *tail_seg, cudaStream_t s) {
    return voxel_reduce<double, false>(perm, seg_off, seg_vox, plan, ntiles, lam, T, logit_prior, E, E, head_part,
                                       tail_part, tail_seg, s);
}

cudaError_t launch_ray_messages_log32(const int64_t *ray_off, int64_t R, const uint32_t *vox, const float *nu,
                                      const float *T, float *lam, float *lbscr, float nu_bg, int first, float L0,
                                      cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    k_ray_messages_log32<<<grid_for(R), kThreads, 0, s>>>(ray_off, R, vox, nu, T, lam, lbscr, nu_bg, first, L0);
    return cudaGetLastError();
}

cudaError_t launch_ray_messages_f64(const int64_t *ray_off, int64_t R, const uint32_t *vox, const double *nu,
                                    const double *T, double *lam, double *bscratch, double nu_bg, int first,
                                    double L0, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    k_ray_messages_f64<<<grid_for(R), kThreads, 0, s>>>(ray_off, R, vox, nu, T, lam, bscratch, nu_bg, first, L0);
    return cudaGetLastError();
}

cudaError_t launch_long_rays_f64(const int64_t *ray_off, const uint32_t *ids, int64_t n_long, const int64_t *loff,
                                 const uint32_t *vox, const float *nu, const float *T, const float *lam, int first,
                                 double L0, double nu_bg, float *out, double *bscr, cudaStream_t s) {
    if (n_long <= 0) return cudaSuccess;
    k_long_rays_f64<<<(unsigned)ceil_div(n_long, 128), 128, 0, s>>>(ray_off, ids, n_long, loff, vox, nu, T, lam, first,
                                                                    L0, nu_bg, out, bscr);
    return cudaGetLastError();
}

cudaError_t launch_long_scatter(const int64_t *ray_off, const uint32_t *ids, int64_t n_long, const int64_t *loff,
                                const float *out, float *lam, cudaStream_t s) {
    if (n_long <= 0) return cudaSuccess;
    k_long_scatter<<<(unsigned)n_long, 32, 0, s>>>(ray_off, ids, n_long, loff, out, lam);
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(float *p, int64_t n, float v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill<float><<<grid_for(n), kThreads, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_fill_f64(double *p, int64_t n, double v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_fill<double><<<grid_for(n), kThreads, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_marginals_f32(const float *T, float *p, GridMap gm, cudaStream_t s) {
    k_marginals<float><<<grid_for((int64_t)gm.nx * gm.ny * gm.nz), kThreads, 0, s>>>(T, p, gm);
    return cudaGetLastError();
}

cudaError_t launch_marginals_f64(const double *T, float *p, GridMap gm, cudaStream_t s) {
    k_marginals<double><<<grid_for((int64_t)gm.nx * gm.ny * gm.nz), kThreads, 0, s>>>(T, p, gm);
    return cudaGetLastError();
}

cudaError_t launch_gather_linear_f32(const float *T, float *out, GridMap gm, cudaStream_t s) {
    k_gather_linear<float><<<grid_for((int64_t)gm.nx * gm.ny * gm.nz), kThreads, 0, s>>>(T, out, gm);
    return cudaGetLastError();
}

cudaError_t launch_gather_linear_f64(const double *T, double *out, GridMap gm, cudaStream_t s) {
    k_gather_linear<double><<<grid_for((int64_t)gm.nx * gm.ny * gm.nz), kThreads, 0, s>>>(T, out, gm);
    return cudaGetLastError();
}

cudaError_t launch_keys_to_linear(const uint32_t *keys, uint32_t *out, int64_t n, GridMap gm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_keys_to_linear<<<grid_for(n), kThreads, 0, s>>>(keys, out, n, gm);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double *a, float *b, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_f64_to_f32<<<grid_for(n), kThreads, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

}  // namespace mrf
