// Per-tile voxel groups, built once per transpose, for the ray kernel's
// pre-aggregation of its messages.
//
// The edges of one ray tile (a run of whole, neighbouring rays) meet the same
// voxels several times: adjacent pixels' rays share most of their voxels.  A
// group is a (tile, voxel) pair.  The ray kernel sums each group's messages in
// shared memory and writes one partial per group, contiguously per tile
// ("tile-major" slots, the tile's groups in voxel order); the voxel totals
// then sum partials instead of messages.  What the kernels need:
//   lidx[q]   for tile-major position q of tile t (q in [E0_t, E1_t)): the
//             window index (edge - base_t) of the q-th edge of t in voxel order
//             (ties in edge order);
//   ends      bit q set when position q ends its group;
//   tg_off[t] the first tile-major slot of tile t;
//   gid[e]    for edge e of tile t: its group's index within the tile (the ray
//             kernel gathers one voxel total per group and reads it by gid);
//   tp2[g]    the tile-major slot of the g-th group in voxel order (tile order
//             within a voxel);
//   seg_off2  voxel segments in group numbering.
// The first four come from one shared-memory sort per tile; tp2 and seg_off2
// from a stable radix sort of the groups' voxel keys (api.cu build_groups).
// The keyframe pairs of the averaging variant are built here as well.
#include "mrf_internal.cuh"

namespace mrf {
namespace {

inline unsigned blocks(int64_t n) { return (unsigned)ceil_div(n > 0 ? n : 1, kThreads); }

// ---- group tables, one CTA per tile.  The tile-major order lists each
// group's positions contiguously, in edge order within a group (so a group's
// partial sum adds its messages in edge order); it writes the window index of
// each position, the group ends and the tile's group count.  Tiles of at most
// 64 rays and 256 distinct bricks take the brick path: the groups are
// numbered in voxel order from per-brick voxel masks (BrickSmem below), and
// per group the set of the tile's rays that cross its voxel (a ray crosses a
// voxel once) gives an edge's rank in its group: the earlier rays in the set.
// Other tiles (many short rays, or rays spread over many bricks)
// sort the tile's edges by (voxel key, window index): a bitonic network over
// 64-bit composites, CAP / 256 per thread in registers (stages within a
// thread in registers, within a warp by shuffles, across warps through shared
// memory).  Either way a tile's groups come in voxel order, which keeps the
// voxel totals' reads of consecutive voxels' partials close together.

using u64 = unsigned long long;

template <typename T, int EPT, int J>
__device__ __forceinline__ void bitonic_in_thread(T (&v)[EPT], int i0, int k) {
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
        if (r & J) continue;
        const T a = v[r], b = v[r + J];
        const bool asc = ((i0 + r) & k) == 0;
        const bool sw = asc ? a > b : a < b;
        v[r] = sw ? b : a;
        v[r + J] = sw ? a : b;
    }
}

// Ascending bitonic sort of the CTA's kThreads * EPT values, EPT per thread in
// blocked order (element i = thread * EPT + r): stages within a thread in
// registers, within a warp by shuffles, across warps through s (as many
// elements).  Every thread of the CTA calls it.
template <typename T, int EPT>
__device__ __forceinline__ void bitonic_block(T (&v)[EPT], T *s) {
    constexpr int N = kThreads * EPT;
    const int i0 = threadIdx.x * EPT;
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= EPT * 32) {   // partner in another warp
                __syncthreads();
#pragma unroll
                for (int r = 0; r < EPT; ++r) s[i0 + r] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < EPT; ++r) {
                    const int i = i0 + r;
                    const T o = s[i ^ j];
                    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                    v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
                }
            } else if (j >= EPT) {   // partner in this warp
                const int lm = j / EPT;
#pragma unroll
                for (int r = 0; r < EPT; ++r) {
                    const int i = i0 + r;
                    const T o = __shfl_xor_sync(0xffffffffu, v[r], lm);
                    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                    v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
                }
            } else if (j == 8) {
                if constexpr (EPT > 8) bitonic_in_thread<T, EPT, 8>(v, i0, k);
            } else if (j == 4) {
                if constexpr (EPT > 4) bitonic_in_thread<T, EPT, 4>(v, i0, k);
            } else if (j == 2) {
                if constexpr (EPT > 2) bitonic_in_thread<T, EPT, 2>(v, i0, k);
            } else {
                if constexpr (EPT > 1) bitonic_in_thread<T, EPT, 1>(v, i0, k);
            }
        }
    }
    __syncthreads();
}

// Sorts s[0, N) ascending in place (N = kThreads * EPT; values past the
// caller's count padded with the largest value).
template <typename T, int EPT>
__device__ __forceinline__ void sort_shared(T *s) {
    T v[EPT];
    const int i0 = threadIdx.x * EPT;
#pragma unroll
    for (int r = 0; r < EPT; ++r) v[r] = s[i0 + r];
    bitonic_block<T, EPT>(v, s);
#pragma unroll
    for (int r = 0; r < EPT; ++r) s[i0 + r] = v[r];
    __syncthreads();
}

// exclusive sum over the CTA's threads, and the total; s_w holds kThreads/32
// words and s_tot one; the barrier inside publishes earlier shared writes
__device__ __forceinline__ uint32_t cta_excl_sum(uint32_t v, uint32_t *s_w, uint32_t *s_tot, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();   // s_w may still be read by an earlier call
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t x = s_w[w];
        before += w < warp ? x : 0u;
        tot += x;
    }
    if (s_tot && threadIdx.x == 0) *s_tot = tot;
    total = tot;
    return before + inc - v;
}

// Bitonic path: sorts the tile and marks the ends in s_bits (tile-local
// positions); returns the group count (valid in thread 0).
template <int CAP>
__device__ __forceinline__ uint32_t tile_groups_sort(int64_t E0, int n, uint32_t off, const uint32_t *vox,
                                                     uint16_t *lidx, uint16_t *gid, uint32_t *gtmp, u64 *s,
                                                     uint32_t *s_bits,
                                                     uint32_t *s_cnt, uint32_t *s_w) {
    constexpr int EPT = CAP / kThreads;
    const int tid = threadIdx.x;
    const int i0 = tid * EPT;
    u64 v[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r)
        v[r] = i0 + r < n ? ((u64)vox[E0 + i0 + r] << 16) | (off + (uint32_t)(i0 + r)) : ~0ull;
    bitonic_block<u64, EPT>(v, s);
    // window indices; the next key for the group ends
    __syncthreads();
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
        s[i0 + r] = v[r];
        if (i0 + r < n) lidx[E0 + i0 + r] = (uint16_t)(v[r] & 0xffffu);
    }
    __syncthreads();
    uint32_t m = 0;   // ends among my EPT positions
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
        const int i = i0 + r;
        const bool end = i < n && (i == n - 1 || (v[r] >> 16) != (s[i + 1] >> 16));
        m |= (uint32_t)end << r;
    }
    if (m) {
        atomicOr(&s_bits[i0 >> 5], m << (i0 & 31));   // i0 is a multiple of EPT: one word
        atomicAdd(s_cnt, (uint32_t)__popc(m));
    }
    // each edge's group index: the ends before its sorted position
    uint32_t tot;
    const uint32_t before = cta_excl_sum((uint32_t)__popc(m), s_w, nullptr, tot);
#pragma unroll
    for (int r = 0; r < EPT; ++r)
        if (i0 + r < n) {
            const uint32_t g = before + (uint32_t)__popc(m & ((1u << r) - 1u));
            gid[E0 + (int64_t)((uint32_t)(v[r] & 0xffffu) - off)] = (uint16_t)g;
            if ((m >> r) & 1u) gtmp[E0 + g] = (uint32_t)(v[r] >> 16);   // the group's voxel key
        }
    __syncthreads();
    return *s_cnt;
}

constexpr uint32_t kEmptyKey = 0xffffffffu;   // voxel keys stay below 2^32 - 1

// shared memory of the brick path (CAP = 2048 edges, 8 per thread).  A voxel
// key is (brick << 9) | Morton index within the 8^3 brick, so voxel order is
// brick order, then Morton order: the tile's distinct bricks are ranked by
// comparison (a few dozen per tile), each brick's voxels are a 512-bit mask,
// and a voxel's group number is its brick's offset plus the set bits below it.
struct BrickSmem {
    static constexpr int kSlots = 1024;   // brick hash table
    static constexpr int kBricks = 256;   // distinct bricks a tile may have on this path
    alignas(16) uint32_t key[kSlots];     // brick of the slot, or empty
    uint16_t bid[kSlots];                 // dense id of the slot's brick
    uint32_t blist[kBricks];              // brick of each dense id
    uint16_t brank[kBricks];              // rank of each dense id in brick order
    alignas(16) uint32_t mask[kBricks * 16];   // by brick rank: the tile's voxels in it, by Morton index
    uint16_t woff[kBricks * 16];          // group number of the first voxel of each mask word
    alignas(16) uint32_t rlo[2048];       // by group: the tile's rays through its voxel (0-31)
    alignas(16) uint32_t rhi[2048];       // (32-63)
    uint16_t goff[2048];                  // by group: its first tile-major position
    uint32_t nb;                          // distinct bricks
};

template <int CAP, bool HASH>
struct TileGroupSmem {
    static constexpr size_t sort_bytes = sizeof(u64) * CAP;
    static constexpr size_t bytes = HASH && sizeof(BrickSmem) > sort_bytes ? sizeof(BrickSmem) : sort_bytes;
};

template <int CAP, bool HASH>
__global__ void __launch_bounds__(kThreads) k_tile_groups(const int64_t *__restrict__ tile_E,
                                                          const uint32_t *__restrict__ hb,
                                                          const uint32_t *__restrict__ vox,
                                                          uint16_t *__restrict__ lidx, uint32_t *__restrict__ ends,
                                                          uint16_t *__restrict__ gid, int32_t *__restrict__ gcount,
                                                          uint32_t *__restrict__ gtmp) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ uint32_t s_bits[CAP / 32 + 2];   // group ends by position within the tile
    __shared__ uint32_t s_w[kThreads / 32];
    __shared__ uint32_t s_cnt;
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x;
    const int64_t E0 = tile_E[t], E1 = tile_E[t + 1];
    const int n = (int)(E1 - E0);   // 1 .. CAP (whole rays packed into the window)
    const uint32_t off = (uint32_t)(E0 & 7);   // window base = E0 rounded down to 8
    if (tid == 0) s_cnt = 0u;
    for (int w = tid; w < CAP / 32 + 2; w += kThreads) s_bits[w] = 0u;
    uint32_t G = 0;
    bool hashed = false;
    if constexpr (HASH) {
        static_assert(CAP == 2048, "brick path: 8 edges per thread");
        BrickSmem &B = *reinterpret_cast<BrickSmem *>(smem_raw);
        // thread tid covers window positions i0 .. i0 + 7 (the window starts at
        // E0 rounded down to 8, so its loads are aligned); vm marks those that
        // are edges of the tile
        const int i0 = tid * 8;
        const int64_t e0t = (E0 & ~(int64_t)7) + i0;
        uint32_t vm = 0;
        {
            const int64_t lo = E0 - e0t, hi = E1 - e0t;
            const int klo = lo < 0 ? 0 : (lo > 8 ? 8 : (int)lo), khi = hi < 0 ? 0 : (hi > 8 ? 8 : (int)hi);
            vm = khi > klo ? ((1u << khi) - 1u) & ~((1u << klo) - 1u) : 0u;
        }
        // ray starts among my edges (the tile's first edge starts a ray); a
        // multiple of 8 never straddles a bitmap word
        const uint32_t sb = vm ? (hb[e0t >> 5] >> (uint32_t)(e0t & 31)) & vm : 0u;
        static_assert(BrickSmem::kSlots == 4 * kThreads, "one 16-byte store per thread clears the table");
        reinterpret_cast<uint4 *>(B.key)[tid] = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
        if (tid == 0) B.nb = 0u;
        uint32_t R = 0;
        const uint32_t rays_before = cta_excl_sum(__popc(sb), s_w, nullptr, R);   // barrier: tables clear
        if (R <= 64) {
            // the tile's bricks, each given a dense id by its first inserter
            // (consecutive edges of a ray mostly share a brick: one insert)
            uint32_t key[8], slot[8], ray[8];
            uint4 k4a = make_uint4(0, 0, 0, 0), k4b = k4a;
            if (vm) {   // 16-byte aligned (the library keeps the keys past the last edge valid)
                k4a = *reinterpret_cast<const uint4 *>(vox + e0t);
                k4b = *reinterpret_cast<const uint4 *>(vox + e0t + 4);
            }
            const uint32_t kw[8] = {k4a.x, k4a.y, k4a.z, k4a.w, k4b.x, k4b.y, k4b.z, k4b.w};
            uint32_t prev_b = kEmptyKey, prev_q = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                key[k] = kEmptyKey;
                slot[k] = 0;
                ray[k] = 0;
                if (!((vm >> k) & 1u)) continue;
                key[k] = kw[k];
                ray[k] = rays_before + __popc(sb & ((2u << k) - 1u)) - 1u;
                const uint32_t b = key[k] >> 9;
                if (b != prev_b) {
                    uint32_t q = (b * 2654435761u) >> 22;   // 10-bit multiplicative hash
                    for (int probe = 0; probe < BrickSmem::kSlots; ++probe) {   // a full table ends the probe
                        const uint32_t old = atomicCAS(&B.key[q], kEmptyKey, b);
                        if (old == kEmptyKey) {
                            const uint32_t id = atomicAdd(&B.nb, 1u);
                            if (id < (uint32_t)BrickSmem::kBricks) {
                                B.blist[id] = b;
                                B.bid[q] = (uint16_t)id;
                            }
                            break;
                        }
                        if (old == b) break;
                        q = (q + 1) & (BrickSmem::kSlots - 1);
                    }
                    prev_b = b;
                    prev_q = q;
                }
                slot[k] = prev_q;
            }
            __syncthreads();
            const uint32_t nb = B.nb;
            if (nb <= (uint32_t)BrickSmem::kBricks) {   // else the sort below
                hashed = true;
                // the bricks' masks start empty (published by the barrier below)
                for (int q = tid; q < (int)nb * 4; q += kThreads) reinterpret_cast<uint4 *>(B.mask)[q] = make_uint4(0, 0, 0, 0);
                // brick ranks: the distinct bricks below each one
                if (tid < (int)nb) {
                    const uint32_t b = B.blist[tid];
                    uint32_t r = 0;
                    for (uint32_t j = 0; j < nb; ++j) r += B.blist[j] < b ? 1u : 0u;
                    B.brank[tid] = (uint16_t)r;
                }
                __syncthreads();
                // the voxel masks; mw = an edge's mask word
                uint32_t mw[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    mw[k] = 0;
                    if (!((vm >> k) & 1u)) continue;
                    const uint32_t low = key[k] & 511u;
                    mw[k] = (uint32_t)B.brank[B.bid[slot[k]]] * 16u + (low >> 5);
                    atomicOr(&B.mask[mw[k]], 1u << (low & 31u));
                }
                __syncthreads();
                // group numbers: per brick (by rank) the voxels before each mask
                // word, then the bricks' offsets
                uint32_t cnt = 0, loc[16];
                if (tid < (int)nb) {
#pragma unroll
                    for (int w = 0; w < 16; ++w) {
                        loc[w] = cnt;
                        cnt += __popc(B.mask[tid * 16 + w]);
                    }
                }
                const uint32_t gbase = cta_excl_sum(cnt, s_w, nullptr, G);
                if (tid < (int)nb) {
#pragma unroll
                    for (int w = 0; w < 16; ++w) B.woff[tid * 16 + w] = (uint16_t)(gbase + loc[w]);
                }
                for (int q = tid; q < (int)(G + 3) / 4; q += kThreads) {   // the groups' ray sets start empty
                    reinterpret_cast<uint4 *>(B.rlo)[q] = make_uint4(0, 0, 0, 0);
                    reinterpret_cast<uint4 *>(B.rhi)[q] = make_uint4(0, 0, 0, 0);
                }
                __syncthreads();
                // each edge's group, and the rays through each group's voxel
                uint32_t grp[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    grp[k] = 0;
                    if (!((vm >> k) & 1u)) continue;
                    const uint32_t low = key[k] & 511u;
                    grp[k] = B.woff[mw[k]] + __popc(B.mask[mw[k]] & ((1u << (low & 31u)) - 1u));
                    atomicOr(ray[k] < 32 ? &B.rlo[grp[k]] : &B.rhi[grp[k]], 1u << (ray[k] & 31u));
                }
                __syncthreads();
                // group offsets: an exclusive scan of the sizes in group order
                uint32_t sz[8], gl = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    sz[k] = i0 + k < (int)G ? __popc(B.rlo[i0 + k]) + __popc(B.rhi[i0 + k]) : 0u;
                    gl += sz[k];
                }
                uint32_t tot;
                uint32_t run = cta_excl_sum(gl, s_w, nullptr, tot);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (i0 + k < (int)G) B.goff[i0 + k] = (uint16_t)run;
                    run += sz[k];
                }
                __syncthreads();
                // rank in the group = earlier rays through the voxel (a ray
                // crosses a voxel once)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (!((vm >> k) & 1u)) continue;
                    const uint32_t lo = B.rlo[grp[k]], hi = B.rhi[grp[k]];
                    const uint32_t rank = ray[k] < 32 ? __popc(lo & ((1u << ray[k]) - 1u))
                                                      : __popc(lo) + __popc(hi & ((1u << (ray[k] - 32u)) - 1u));
                    const uint32_t pos = B.goff[grp[k]] + rank;
                    lidx[E0 + pos] = (uint16_t)(i0 + k);   // the window index
                    if (rank == 0) gtmp[E0 + grp[k]] = key[k];   // the group's voxel key
                    if (vm != 0xffu) gid[e0t + k] = (uint16_t)grp[k];
                    if (rank + 1 == (uint32_t)(__popc(lo) + __popc(hi))) atomicOr(&s_bits[pos >> 5], 1u << (pos & 31));
                }
                if (vm == 0xffu)   // all eight group indices in one 16-byte store
                    *reinterpret_cast<uint4 *>(gid + e0t) =
                        make_uint4(grp[0] | (grp[1] << 16), grp[2] | (grp[3] << 16), grp[4] | (grp[5] << 16),
                                   grp[6] | (grp[7] << 16));
                __syncthreads();
            }
        }
    }
    if (!hashed) {
        __syncthreads();
        G = tile_groups_sort<CAP>(E0, n, off, vox, lidx, gid, gtmp, reinterpret_cast<u64 *>(smem_raw), s_bits, &s_cnt,
                                  s_w);
    }
    // to the global bitmap: word w holds positions [32 w, 32 w + 32); words
    // shared with neighbouring tiles are OR-ed in
    const int64_t w0 = E0 >> 5, w1 = (E1 - 1) >> 5;
    for (int64_t w = w0 + tid; w <= w1; w += kThreads) {
        const int64_t lb = (w << 5) - E0;   // tile-local position of bit 0 (may be negative)
        const int64_t q = lb >> 5;          // floor division (arithmetic shift)
        const uint32_t sh = (uint32_t)(lb & 31);
        const uint32_t a = q >= 0 ? s_bits[q] : 0u;
        const uint32_t b = q + 1 >= 0 ? s_bits[q + 1] : 0u;
        const uint32_t bits = (uint32_t)((((u64)b << 32) | a) >> sh);
        if (w == w0 || w == w1) {
            if (bits) atomicOr(&ends[w], bits);
        } else {
            ends[w] = bits;
        }
    }
    if (tid == 0) gcount[t] = (int32_t)G;
}

// The voxel key of every group, by slot: tile t's group keys, written by the
// tile-groups kernel at gtmp[tile_E[t] + g], moved to gkey[tg_off[t] + g]; a
// warp per tile.
__global__ void __launch_bounds__(kThreads) k_group_keys(const int64_t *__restrict__ tile_E, int64_t ntiles,
                                                         const int64_t *__restrict__ tg_off,
                                                         const uint32_t *__restrict__ gtmp, uint32_t *__restrict__ gkey) {
    const int64_t t = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    const int64_t E0 = tile_E[t], g0 = tg_off[t];
    const int ng = (int)(tg_off[t + 1] - g0);
    for (int g = threadIdx.x & 31; g < ng; g += 32) gkey[g0 + g] = gtmp[E0 + g];
}

// ---- per-keyframe average messages (the implementation's Section "Belief
// Propagation"): all rays of one keyframe through a voxel send the mean of
// their messages.  Frames own contiguous edge ranges and the transpose is
// stable, so within a voxel's run of the voxel-major order each frame's edges
// are contiguous: a (frame, voxel) pair is a run of equal (voxel, frame).

__device__ __forceinline__ int32_t frame_of(const int64_t *frame_E, int32_t n_frames, int64_t e) {
    int32_t lo = 0, hi = n_frames - 1;   // the last frame whose first edge is <= e
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (frame_E[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_pair_flags(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ vox, int64_t E,
                             const int64_t *__restrict__ frame_E, int32_t n_frames, int32_t *__restrict__ flags) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= E) return;
    const uint32_t e = perm[k];
    int32_t f = 1;
    if (k > 0) {
        const uint32_t q = perm[k - 1];
        f = vox[e] != vox[q] || frame_of(frame_E, n_frames, e) != frame_of(frame_E, n_frames, q);
    }
    flags[k] = f;
}

// pair offsets, the pair of every voxel-major position, and the identity map
// the segmented reduction writes the pair sums through
__global__ void k_pair_starts(const int32_t *__restrict__ flags, const int64_t *__restrict__ pos, int64_t E,
                              uint32_t *__restrict__ pair_off, uint32_t *__restrict__ pid,
                              uint32_t *__restrict__ ident) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= E) return;
    pid[k] = (uint32_t)(pos[k] + flags[k] - 1);
    if (flags[k]) {
        pair_off[pos[k]] = (uint32_t)k;
        ident[pos[k]] = (uint32_t)pos[k];
    }
    if (k == 0) pair_off[pos[E]] = (uint32_t)E;
}

// every edge of a pair gets the pair's mean (sums from the fixed-order
// segmented reduction, so the result is reproducible)
__global__ void k_pair_scatter(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ pid,
                               const uint32_t *__restrict__ pair_off, const float *__restrict__ sums, int64_t E,
                               float *__restrict__ lam) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= E) return;
    const uint32_t p = pid[k];
    lam[perm[k]] = sums[p] / (float)(pair_off[p + 1] - pair_off[p]);
}

}  // namespace

cudaError_t launch_tile_sort(int cap, const int64_t *tile_E, int64_t ntiles, const uint32_t *hb, const uint32_t *vox,
                             uint16_t *lidx, uint32_t *ends, uint16_t *gid, int32_t *gcount, uint32_t *gtmp,
                             cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (cap == 2048) {
        constexpr int bytes = (int)TileGroupSmem<2048, true>::bytes;
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute(k_tile_groups<2048, true>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        k_tile_groups<2048, true><<<(unsigned)ntiles, kThreads, bytes, s>>>(tile_E, hb, vox, lidx, ends, gid, gcount,
                                                                                  gtmp);
    } else if (cap == 4096) {
        constexpr int bytes = (int)TileGroupSmem<4096, false>::bytes;
        k_tile_groups<4096, false><<<(unsigned)ntiles, kThreads, bytes, s>>>(tile_E, hb, vox, lidx, ends, gid, gcount,
                                                                                  gtmp);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
cudaError_t launch_group_keys(const int64_t *tile_E, int64_t ntiles, const int64_t *tg_off, const uint32_t *gtmp,
                              uint32_t *gkey, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_group_keys<<<(unsigned)ceil_div(ntiles, kThreads / 32), kThreads, 0, s>>>(tile_E, ntiles, tg_off, gtmp, gkey);
    return cudaGetLastError();
}
cudaError_t launch_pair_flags(const uint32_t *perm, const uint32_t *vox, int64_t E, const int64_t *frame_E,
                              int32_t n_frames, int32_t *flags, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    k_pair_flags<<<blocks(E), kThreads, 0, s>>>(perm, vox, E, frame_E, n_frames, flags);
    return cudaGetLastError();
}
cudaError_t launch_pair_starts(const int32_t *flags, const int64_t *pos, int64_t E, uint32_t *pair_off,
                               uint32_t *pid, uint32_t *ident, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    k_pair_starts<<<blocks(E), kThreads, 0, s>>>(flags, pos, E, pair_off, pid, ident);
    return cudaGetLastError();
}
cudaError_t launch_pair_scatter(const uint32_t *perm, const uint32_t *pid, const uint32_t *pair_off,
                                const float *sums, int64_t E, float *lam, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    k_pair_scatter<<<blocks(E), kThreads, 0, s>>>(perm, pid, pair_off, sums, E, lam);
    return cudaGetLastError();
}

}  // namespace mrf
