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
//   tp2[g]    the tile-major slot of the g-th group in voxel order (tile order
//             within a voxel);
//   seg_off2  voxel segments in group numbering.
// The first three come from one shared-memory sort per tile; tp2 and seg_off2
// from a stable radix sort of the groups' voxel keys (api.cu build_groups).
// The keyframe pairs of the averaging variant are built here as well.
#include "mrf_internal.cuh"

namespace mrf {
namespace {

inline unsigned blocks(int64_t n) { return (unsigned)ceil_div(n > 0 ? n : 1, kThreads); }

// ---- group tables by a per-tile sort.  One CTA per tile sorts the tile's
// edges by (voxel key, window index) (a bitonic network over 64-bit
// composites, CAP / 256 per thread in registers: stages within a thread in
// registers, within a warp by shuffles, across warps through shared memory),
// which is the tile-major order itself: position E0 + i of the tile holds its
// i-th smallest (voxel, edge).  It writes the window index of each position,
// the group ends (last position of each voxel's run) and the tile's group
// count.

using u64 = unsigned long long;

template <int EPT, int J>
__device__ __forceinline__ void bitonic_in_thread(u64 (&v)[EPT], int i0, int k) {
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
        if (r & J) continue;
        const u64 a = v[r], b = v[r + J];
        const bool asc = ((i0 + r) & k) == 0;
        const bool sw = asc ? a > b : a < b;
        v[r] = sw ? b : a;
        v[r + J] = sw ? a : b;
    }
}

template <int CAP>
__global__ void __launch_bounds__(kThreads) k_tile_sort(const int64_t *__restrict__ tile_E,
                                                        const uint32_t *__restrict__ vox, uint16_t *__restrict__ lidx,
                                                        uint32_t *__restrict__ ends, int32_t *__restrict__ gcount) {
    constexpr int EPT = CAP / kThreads;   // 8 or 16 elements per thread
    __shared__ u64 s[CAP];
    __shared__ uint32_t s_bits[CAP / 32 + 2];   // group ends by position within the tile
    __shared__ uint32_t s_cnt;
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x;
    const int64_t E0 = tile_E[t], E1 = tile_E[t + 1];
    const int n = (int)(E1 - E0);   // 1 .. CAP (whole rays packed into the window)
    const uint32_t off = (uint32_t)(E0 & 7);   // window base = E0 rounded down to 8
    const int i0 = tid * EPT;
    if (tid == 0) s_cnt = 0u;
    for (int w = tid; w < CAP / 32 + 2; w += kThreads) s_bits[w] = 0u;
    u64 v[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r)
        v[r] = i0 + r < n ? ((u64)vox[E0 + i0 + r] << 16) | (off + (uint32_t)(i0 + r)) : ~0ull;
    for (int k = 2; k <= CAP; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= EPT * 32) {   // partner in another warp
                __syncthreads();
#pragma unroll
                for (int r = 0; r < EPT; ++r) s[i0 + r] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < EPT; ++r) {
                    const int i = i0 + r;
                    const u64 o = s[i ^ j];
                    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                    v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
                }
            } else if (j >= EPT) {   // partner in this warp
                const int lm = j / EPT;
#pragma unroll
                for (int r = 0; r < EPT; ++r) {
                    const int i = i0 + r;
                    const u64 o = __shfl_xor_sync(0xffffffffu, v[r], lm);
                    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                    v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
                }
            } else if (j == 8) {
                if constexpr (EPT > 8) bitonic_in_thread<EPT, 8>(v, i0, k);
            } else if (j == 4) {
                bitonic_in_thread<EPT, 4>(v, i0, k);
            } else if (j == 2) {
                bitonic_in_thread<EPT, 2>(v, i0, k);
            } else {
                bitonic_in_thread<EPT, 1>(v, i0, k);
            }
        }
    }
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
        atomicAdd(&s_cnt, (uint32_t)__popc(m));
    }
    __syncthreads();
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
    if (tid == 0) gcount[t] = (int32_t)s_cnt;
}

// The voxel key of every group, by slot (tile offset + rank of the group's end
// among the tile's ends).
__global__ void __launch_bounds__(kThreads) k_group_keys(const int64_t *__restrict__ tile_E,
                                                         const int64_t *__restrict__ tg_off,
                                                         const uint32_t *__restrict__ ends,
                                                         const uint16_t *__restrict__ lidx,
                                                         const uint32_t *__restrict__ vox, uint32_t *__restrict__ gkey) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const int64_t t = blockIdx.x;
    const int64_t E0 = tile_E[t], E1 = tile_E[t + 1];
    const int64_t base = E0 & ~(int64_t)7;
    const int64_t w = (E0 >> 5) + threadIdx.x;   // a tile spans at most CAP / 32 + 2 <= 130 words
    uint32_t bits = 0;
    if (w <= ((E1 - 1) >> 5)) {
        bits = ends[w];
        const int64_t lo = E0 - (w << 5), hi = E1 - (w << 5);   // keep bits [lo, hi)
        if (lo > 0) bits &= ~0u << (uint32_t)lo;
        if (hi < 32) bits &= (1u << (uint32_t)hi) - 1u;
    }
    // exclusive count of ends over the threads
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t c = __popc(bits);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t before = inc - c;
    for (int i = 0; i < warp; ++i) before += s_warp[i];
    uint32_t *out = gkey + tg_off[t] + before;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        *out++ = vox[base + lidx[(w << 5) + b]];
    }
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

cudaError_t launch_tile_sort(int cap, const int64_t *tile_E, int64_t ntiles, const uint32_t *vox, uint16_t *lidx,
                             uint32_t *ends, int32_t *gcount, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (cap == 2048) k_tile_sort<2048><<<(unsigned)ntiles, kThreads, 0, s>>>(tile_E, vox, lidx, ends, gcount);
    else if (cap == 4096) k_tile_sort<4096><<<(unsigned)ntiles, kThreads, 0, s>>>(tile_E, vox, lidx, ends, gcount);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
cudaError_t launch_group_keys(const int64_t *tile_E, int64_t ntiles, const int64_t *tg_off, const uint32_t *ends,
                              const uint16_t *lidx, const uint32_t *vox, uint32_t *gkey, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_group_keys<<<(unsigned)ntiles, kThreads, 0, s>>>(tile_E, tg_off, ends, lidx, vox, gkey);
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
