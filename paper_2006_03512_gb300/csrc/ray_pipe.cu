// Ray -> voxel messages for the context's own (padded) edge arrays: a
// persistent, software-pipelined version of the per-tile computation in
// ray_tile.cuh.
//
// Each CTA owns a contiguous range of ray tiles (neighbouring rays, so their
// voxels and the T entries they gather overlap).  Two shared-memory stages
// hold a tile's voxel keys, likelihoods and old messages; the next tile's
// stage is filled by TMA bulk copies (cp.async.bulk, completion on an mbarrier)
// issued when the current tile starts.  Half-way through the current tile
// (after its CTA-wide scans) the threads wait for that copy and each gathers
// the voxel totals T[key] of its own edges of the next tile with cp.async,
// together with the words of the ray-start bitmap it needs; those land while
// the current tile finishes.  Two stages keep shared memory at ~68 KB, so three
// CTAs fit on an SM.
//
// Every mbarrier wait is bounded; a wait that gives up sets bit 1 of *err, and
// the CTA leaves after all threads agree (no thread is left at a barrier).
#include <cuda_bf16.h>

#include <type_traits>

#include "mrf_internal.cuh"
#include "ray_tile.cuh"

namespace mrf {
namespace {

using tile::Bwd;
using tile::Fwd;

// A wait gives up after kWaitNs of the global timer (the copies it waits for
// take microseconds), or after kWaitLimit polls, whichever comes first.
constexpr uint32_t kWaitLimit = 1u << 26;
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// the timed part of a wait that the first polls did not end (out of line, so
// that the kernels' common path stays a plain polling loop)
__device__ __noinline__ bool mbar_wait_timed(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 256u; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// bounded wait; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < 256u; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait_timed(bar, parity);
}

// Exclusive sum of v over the CTA's NT threads (v >= 0).  The barrier inside
// also publishes every shared-memory write made before the call.
template <int NT>
__device__ __forceinline__ int block_count_exclusive(int v, int *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    constexpr int NW = NT / 32;
    int t = lane < NW ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
    }
    const int pre = __shfl_sync(0xffffffffu, t, (warp + 31) & 31);
    return (warp ? pre : 0) + inc - v;
}

// Per-edge messages are stored as FP32, or as bf16 (rounded to nearest even;
// the arithmetic is FP32 either way).
template <typename LamT>
__host__ __device__ constexpr bool is_bf16() { return std::is_same<LamT, __nv_bfloat16>::value; }

template <int KT, int NT, typename LamT>
struct PipeSmem {
    static constexpr int CAP = NT * KT;
    uint32_t vox[2][CAP];
    float nu[2][CAP];
    LamT lam[2][CAP];
    float T[2][CAP];          // gathered voxel totals; then the tile's messages by window index
    uint16_t lx[2][CAP];      // grouping: window index of each tile-major position
    int64_t E0[2], E1[2], tg[2];
    uint64_t bar[2];
    Fwd fw[NT / 32];
    Bwd bw[NT / 32];
    int cnt[NT / 32];         // group ends per warp
    float2 tail[NT];          // per thread: sum after its last group end, and whether it has one
};

// First edge of a tile's 256*KT-edge window (aligned to 8 edges).
__device__ __forceinline__ int64_t window_base(int64_t E0) { return E0 & ~(int64_t)7; }

// Resident CTAs per SM the register budget is set for: three for 2048-edge
// tiles (about 76 KB of shared memory each), one otherwise.
template <int KT, int NT>
constexpr int pipe_min_blocks() { return NT * KT == 2048 ? (NT >= 512 ? 2 : 3) : 1; }

template <int KT, bool AGG, int NT, typename LamT, bool FL>
__global__ void __launch_bounds__(NT, pipe_min_blocks<KT, NT>())
    k_ray_pipe(const int64_t *__restrict__ tile_E, int64_t ntiles, const uint32_t *__restrict__ hb,
               const uint32_t *__restrict__ vox, const float *__restrict__ nu, const float *__restrict__ T,
               LamT *__restrict__ lam, float nu_bg, float nu_ref, int first, float L0, uint32_t *__restrict__ err,
               const uint16_t *__restrict__ lidx, const uint32_t *__restrict__ ends,
               const int64_t *__restrict__ tg_off, float *__restrict__ partial) {
    using S = PipeSmem<KT, NT, LamT>;
    constexpr int CAP = S::CAP;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * ntiles / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * ntiles / gridDim.x;
    const int n = (int)(t1 - t0);
    if (n <= 0) return;
    const uint32_t stage_bytes = (uint32_t)(CAP * 4) + (first ? 0u : (uint32_t)(CAP * (4 + sizeof(LamT))));

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) mbar_init(&sm.bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0: bulk copies of tile j into stage j % 2
    auto issue = [&](int j) {
        const int st = j & 1;
        const int64_t E0 = tile_E[t0 + j], E1 = tile_E[t0 + j + 1];
        const int64_t base = window_base(E0);
        sm.E0[st] = E0;
        sm.E1[st] = E1;
        if (AGG) sm.tg[st] = tg_off[t0 + j];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&sm.bar[st], stage_bytes);
        tma_load_1d(sm.nu[st], nu + base, CAP * 4, &sm.bar[st]);
        if (!first) {
            tma_load_1d(sm.vox[st], vox + base, CAP * 4, &sm.bar[st]);
            tma_load_1d(sm.lam[st], lam + base, CAP * (uint32_t)sizeof(LamT), &sm.bar[st]);
        }
    };
    // every thread, once tile j's keys are in: cp.async of its own T entries
    // (and, when grouping, of its 8-edge slice of the tile-major order), and
    // plain loads of the bitmap words covering its edges
    // a thread's KT bits start at a multiple of 8 within a word, so with KT > 8
    // they can straddle two words
    constexpr bool kEnds2 = KT > 8;
    uint32_t hw0 = 0, hw1 = 0, ew0 = 0, ew1 = 0;   // for the tile being computed
    uint32_t nh0 = 0, nh1 = 0, ne0 = 0, ne1 = 0;   // for the next one
    auto gather = [&](int j) {
        const int st = j & 1;
        const int64_t E0 = sm.E0[st], E1 = sm.E1[st];
        const int64_t base = window_base(E0);
        const int64_t my0 = base + (int64_t)tid * KT;
        const int64_t w = my0 >> 5;
        nh0 = hb[w];
        nh1 = hb[w + 1];
        if (AGG) {
            ne0 = ends[w];
            if (kEnds2) ne1 = ends[w + 1];
            if constexpr (KT % 8 == 0) {
#pragma unroll
                for (int k = 0; k < KT; k += 8)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                     smem_u32(&sm.lx[st][tid * KT + k])),
                                 "l"(lidx + my0 + k)
                                 : "memory");
            } else {   // KT = 4: 8 bytes, aligned since my0 is a multiple of 4
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.lx[st][tid * KT])),
                             "l"(lidx + my0)
                             : "memory");
            }
        }
        if (!first) {
            // a warp gathers the T entries of its own threads' edges, lane l
            // taking every 32nd edge from l: neighbouring edges of a ray share
            // cache sectors, so a warp-wide gather touches fewer of them
            const int i0 = (int)(E0 - base), i1 = (int)(E1 - base);
            const int wb = (tid & ~31) * KT + (tid & 31);
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                const int i = wb + k * 32;
                if (i >= i0 && i < i1) cp_async4(&sm.T[st][i], T + sm.vox[st][i]);
            }
        }
        cp_async_commit();
    };
    auto leave_on_timeout = [&](bool ok) {
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, 2u);
            return true;
        }
        return false;
    };

    if (tid == 0) issue(0);
    __syncthreads();
    if (leave_on_timeout(mbar_wait(&sm.bar[0], 0))) return;
    gather(0);

    bool timed_out = false;
    for (int j = 0; j < n; ++j) {
        const int st = j & 1;
        if (tid == 0 && j + 1 < n) issue(j + 1);
        cp_async_wait<0>();   // this thread's copies for tile j
        __syncwarp();         // and those of the other lanes (T entries of this warp's edges)
        hw0 = nh0;
        hw1 = nh1;
        ew0 = ne0;
        ew1 = ne1;
        // the stage's scalars are read before the tile's first barrier: thread 0
        // refills this stage's slots when it starts tile j + 1, which it can do
        // once every thread has passed the tile's last barrier
        const int64_t E0 = sm.E0[st], E1 = sm.E1[st];
        const int64_t tg = AGG ? sm.tg[st] : 0;
        const int64_t base = window_base(E0);
        const int64_t my0 = base + (int64_t)tid * KT;
        const uint32_t vmask = tile::valid_mask<KT>(my0, E0, E1);
        const uint32_t bmask = KT == 32 ? 0xffffffffu : ((1u << KT) - 1u);
        // ray starts among my edges, and ends: an edge ends a ray when the
        // next edge starts one or it is the tile's last edge
        const uint64_t words = ((uint64_t)hw1 << 32) | hw0;
        const uint64_t bits = words >> (uint32_t)(my0 & 31);
        const uint32_t hbits = (uint32_t)bits & bmask & vmask;
        uint32_t tbits = (uint32_t)(bits >> 1) & bmask;
        const int64_t last = E1 - 1 - my0;
        if (last >= 0 && last < KT) tbits |= 1u << (uint32_t)last;
        tbits &= vmask;
        float nv[KT], lo[KT];
#pragma unroll
        for (int k = 0; k < KT; k += 4) {
            const float4 n4 = *reinterpret_cast<const float4 *>(&sm.nu[st][tid * KT + k]);
            nv[k] = n4.x; nv[k + 1] = n4.y; nv[k + 2] = n4.z; nv[k + 3] = n4.w;
        }
        if (first) {
#pragma unroll
            for (int k = 0; k < KT; ++k) lo[k] = L0;
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
                const float4 g4 = *reinterpret_cast<const float4 *>(&sm.T[st][tid * KT + k]);
                lo[k] = g4.x - l4.x; lo[k + 1] = g4.y - l4.y; lo[k + 2] = g4.z - l4.z; lo[k + 3] = g4.w - l4.w;
            }
        }
        // half-way: the next tile's copy has had the scans' time to land
        auto mid = [&]() {
            if (j + 1 < n) {
                const bool ok = mbar_wait(&sm.bar[(j + 1) & 1], ((j + 1) >> 1) & 1);
                if (__syncthreads_or(!ok)) {
                    timed_out = true;
                    return;
                }
                gather(j + 1);
            }
        };
        tile::tile_messages<KT, NT, FL>(nv, lo, vmask, hbits, tbits, nu_bg, nu_ref, sm.fw, sm.bw, mid);
        if (timed_out) {
            if (tid == 0) atomicOr(err, 2u);
            cp_async_wait<0>();
            return;
        }
        if constexpr (is_bf16<LamT>()) {
            // store the rounded messages; the voxel totals below sum the same
            // rounded values, so the next cavity removes exactly what was added
            uint32_t hb16[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                hb16[k] = __bfloat16_as_ushort(__float2bfloat16_rn(nv[k]));
                nv[k] = __uint_as_float(hb16[k] << 16);
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
                    *reinterpret_cast<float4 *>(lam + my0 + k) = make_float4(nv[k], nv[k + 1], nv[k + 2], nv[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < KT; ++k)
                    if ((vmask >> k) & 1u) lam[my0 + k] = nv[k];
            }
        }
        if (AGG) {
            // One partial sum per (tile, voxel) group.  The tile's messages go to
            // shared memory by window index (over the gathered T values, no longer
            // needed); position q of the tile's voxel order reads its message
            // through lx.  Each thread publishes the sum of its positions after
            // its last group end (all of them if it has none); the thread holding
            // a group's end adds those of the earlier threads back to the one
            // where the group began, then its own positions.  Group g of the
            // tile (in voxel order) lands in slot tg + g.
            float *sl = sm.T[st];
            if (vmask == bmask) {
#pragma unroll
                for (int k = 0; k < KT; k += 4)
                    *reinterpret_cast<float4 *>(&sl[tid * KT + k]) = make_float4(nv[k], nv[k + 1], nv[k + 2], nv[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < KT; ++k)
                    if ((vmask >> k) & 1u) sl[tid * KT + k] = nv[k];
            }
            const uint32_t ebits =
                (uint32_t)((((uint64_t)ew1 << 32) | ew0) >> (uint32_t)(my0 & 31)) & bmask & vmask;
            __syncthreads();
            const uint16_t *lxs = sm.lx[st];
            float x[KT];
#pragma unroll
            for (int k = 0; k < KT; k += 4) {
                const uint2 w2 = *reinterpret_cast<const uint2 *>(&lxs[tid * KT + k]);
                const uint32_t wv[2] = {w2.x, w2.y};
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    x[k + 2 * i] = ((vmask >> (k + 2 * i)) & 1u) ? sl[wv[i] & 0xffffu] : 0.f;
                    x[k + 2 * i + 1] = ((vmask >> (k + 2 * i + 1)) & 1u) ? sl[wv[i] >> 16] : 0.f;
                }
            }
            float tl = 0.f;
#pragma unroll
            for (int k = 0; k < KT; ++k) tl = ((ebits >> k) & 1u) ? 0.f : tl + x[k];
            sm.tail[tid] = make_float2(tl, ebits ? 1.f : 0.f);
            const int before = block_count_exclusive<NT>(__popc(ebits), sm.cnt);   // barrier: tails are in
            if (ebits) {
                float acc = 0.f;
                for (int t = tid - 1; t >= 0; --t) {
                    const float2 e = sm.tail[t];
                    acc += e.x;
                    if (e.y != 0.f) break;
                }
                float *out = partial + tg + before;
#pragma unroll
                for (int k = 0; k < KT; ++k) {
                    acc += x[k];
                    if ((ebits >> k) & 1u) {
                        *out++ = acc;
                        acc = 0.f;
                    }
                }
            }
        }
        // no barrier here: the next tile's first barrier (in its scans) comes
        // before anything that overwrites what this tile still reads
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
                        const uint16_t *lidx, const uint32_t *ends, const int64_t *tg_off, float *partial,
                        cudaStream_t s) {
    static int per_sm = 0;   // resident CTAs per SM, from the occupancy calculator
    const int bytes = (int)sizeof(PipeSmem<KT, NT, LamT>);
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
        tile_E, ntiles, hb, vox, nu, T, static_cast<LamT *>(lam), nu_bg, nu_ref, first, L0, err, lidx, ends, tg_off,
        partial);
    return cudaGetLastError();
}

}  // namespace

bool ray_pipe_supported(int kt, int nt) {
    return (nt == kThreads && (kt == 8 || kt == 16)) || (nt == 128 && kt == 16) || (nt == 512 && kt == 4);
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
                            const uint32_t *ends, const int64_t *tg_off, float *partial, cudaStream_t s,
                            bool floored) {
    if (ntiles <= 0) return cudaSuccess;
    const bool agg = partial != nullptr;
    if (bf16 && !agg) return cudaErrorInvalidValue;   // bf16 storage is for the grouped path only
#define MRF_PIPE(KT, AGG, NT, LT)                                                                                   \
    return launch_pipe<KT, AGG, NT, LT>(n_sm, tile_E, ntiles, hb, vox, nu, T, lam, nu_bg, nu_ref, first, L0, err,   \
                                        lidx, ends, tg_off, partial, s)
#define MRF_PIPE_FL(KT, AGG, NT, LT)                                                                                \
    return launch_pipe<KT, AGG, NT, LT, true>(n_sm, tile_E, ntiles, hb, vox, nu, T, lam, nu_bg, nu_ref, first, L0,  \
                                              err, lidx, ends, tg_off, partial, s)
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
