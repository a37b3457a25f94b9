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
// edges by (voxel key, window index) in shared memory (bitonic network over
// 64-bit composites), which is the tile-major order itself: position E0 + i
// of the tile holds its i-th smallest (voxel, edge).  It writes the window
// index of each position, the group ends (last position of each voxel's run)
// and the tile's group count.

template <int CAP>
__global__ void __launch_bounds__(kThreads) k_tile_sort(const int64_t *__restrict__ tile_E,
                                                        const uint32_t *__restrict__ vox, uint16_t *__restrict__ lidx,
                                                        uint32_t *__restrict__ ends, int32_t *__restrict__ gcount) {
    __shared__ unsigned long long s[CAP];
    __shared__ uint32_t s_cnt;
    const int64_t t = blockIdx.x;
    const int64_t E0 = tile_E[t], E1 = tile_E[t + 1];
    const int n = (int)(E1 - E0);   // 1 .. CAP (whole rays packed into the window)
    const uint32_t off = (uint32_t)(E0 & 7);   // window base = E0 rounded down to 8
    int np = 1;
    while (np < n) np <<= 1;
    if (threadIdx.x == 0) s_cnt = 0u;
    for (int i = threadIdx.x; i < np; i += kThreads)
        s[i] = i < n ? ((unsigned long long)vox[E0 + i] << 16) | (off + (uint32_t)i) : ~0ull;
    __syncthreads();
    for (int k = 2; k <= np; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < (np >> 1); q += kThreads) {
                const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                const unsigned long long a = s[i], b = s[i + j];
                if ((a > b) == ((i & k) == 0)) {
                    s[i] = b;
                    s[i + j] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += kThreads) lidx[E0 + i] = (uint16_t)(s[i] & 0xffffu);
    // group ends: one bitmap word per thread (words at the tile's edges are
    // shared with the neighbouring tiles, hence the atomic OR)
    uint32_t cnt = 0;
    for (int64_t w = (E0 >> 5) + threadIdx.x; w <= ((E1 - 1) >> 5); w += kThreads) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t pos = (w << 5) + b;
            if (pos < E0 || pos >= E1) continue;
            const int i = (int)(pos - E0);
            if (i == n - 1 || (s[i] >> 16) != (s[i + 1] >> 16)) bits |= 1u << b;
        }
        if (bits) atomicOr(&ends[w], bits);
        cnt += __popc(bits);
    }
    if (cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) gcount[t] = (int32_t)s_cnt;
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
