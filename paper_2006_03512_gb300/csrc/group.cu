// Per-tile voxel groups, built once per transpose, for the ray kernel's
// pre-aggregation of its messages.
//
// The edges of one ray tile (a run of whole, neighbouring rays) meet the same
// voxels several times: adjacent pixels' rays share most of their voxels.  A
// group is a (tile, voxel) pair.  Because the voxel-sorted edge list is stable
// by edge id and tiles are contiguous edge ranges, each group is a contiguous
// run of that list; the groups are numbered in that order (gid).  The ray
// kernel sums each group's messages in shared memory and writes one partial
// per group, contiguously per tile ("tile-major" slots); the voxel totals then
// sum partials instead of messages.  What the kernels need:
//   lidx[q]   for tile-major position q of tile t (q in [E0_t, E1_t)): the
//             window index (edge - base_t) of the q-th edge of t in voxel order;
//   ends      bit q set when position q ends its group;
//   tg_off[t] the first tile-major slot of tile t;
//   tp2[g]    the tile-major slot of group g (voxel order -> slot);
//   seg_off2  voxel segments in group numbering.
#include "mrf_internal.cuh"

namespace mrf {
namespace {

__global__ void k_tile_ids(const int64_t *__restrict__ tile_E, uint32_t *__restrict__ tid_of) {
    const int64_t t = blockIdx.x;
    const int64_t e0 = tile_E[t], e1 = tile_E[t + 1];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) tid_of[e] = (uint32_t)t;
}

__global__ void k_tile_keys(const uint32_t *__restrict__ perm, int64_t E, const uint32_t *__restrict__ tid_of,
                            uint32_t *__restrict__ tkey) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < E) tkey[k] = tid_of[perm[k]];
}

// a group starts at sorted position k when the voxel or the tile changes
__global__ void k_group_starts(const uint32_t *__restrict__ vkey, const uint32_t *__restrict__ tkey, int64_t E,
                               uint32_t *__restrict__ flags) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < E) flags[k] = (k == 0 || vkey[k] != vkey[k - 1] || tkey[k] != tkey[k - 1]) ? 1u : 0u;
}

// gid[k] = (number of group starts in [0, k]) - 1, from the exclusive scan
__global__ void k_group_ids(const uint32_t *__restrict__ starts, const uint32_t *__restrict__ excl, int64_t E,
                            uint32_t *__restrict__ gid) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < E) gid[k] = excl[k] + starts[k] - 1u;
}

// tile-major position q -> local window index, group end bits and start flags
__global__ void k_tile_major(const uint32_t *__restrict__ tperm, const uint32_t *__restrict__ perm,
                             const uint32_t *__restrict__ gid, const int64_t *__restrict__ tile_E,
                             const uint32_t *__restrict__ tid_of, int64_t E, uint16_t *__restrict__ lidx,
                             uint32_t *__restrict__ ends, uint32_t *__restrict__ tstart) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool end = false;
    if (q < E) {
        const uint32_t t = tid_of[q];
        const int64_t E0 = tile_E[t], E1 = tile_E[t + 1];
        const int64_t base = E0 & ~(int64_t)7;
        const uint32_t k = tperm[q];
        const uint32_t g = gid[k];
        lidx[q] = (uint16_t)((int64_t)perm[k] - base);
        end = (q == E1 - 1) || gid[tperm[q + 1]] != g;
        tstart[q] = (q == E0 || gid[tperm[q - 1]] != g) ? 1u : 0u;
    }
    // positions are numbered from a multiple of 32 per warp, so each warp owns one word
    const uint32_t word = __ballot_sync(0xffffffffu, end);
    if ((threadIdx.x & 31) == 0 && q < E) ends[q >> 5] = word;
}

__global__ void k_group_slots(const uint32_t *__restrict__ tperm, const uint32_t *__restrict__ gid,
                              const uint32_t *__restrict__ tstart, const uint32_t *__restrict__ tmi,
                              const int64_t *__restrict__ tile_E, const uint32_t *__restrict__ tid_of,
                              int64_t ntiles, int64_t E, uint32_t *__restrict__ tp2, int64_t *__restrict__ tg_off) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= E) return;
    if (tstart[q]) tp2[gid[tperm[q]]] = tmi[q];
    const uint32_t t = tid_of[q];
    if (tile_E[t] == q) tg_off[t] = tmi[q];
    if (q == 0) tg_off[ntiles] = tmi[E];
}

__global__ void k_seg_groups(const uint32_t *__restrict__ seg_off, int64_t S, const uint32_t *__restrict__ gid,
                             int64_t G, uint32_t *__restrict__ seg_off2) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) seg_off2[s] = gid[seg_off[s]];
    if (s == S) seg_off2[S] = (uint32_t)G;
}

inline unsigned blocks(int64_t n) { return (unsigned)ceil_div(n > 0 ? n : 1, kThreads); }

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

cudaError_t launch_tile_ids(const int64_t *tile_E, int64_t ntiles, uint32_t *tid_of, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_tile_ids<<<(unsigned)ntiles, kThreads, 0, s>>>(tile_E, tid_of);
    return cudaGetLastError();
}
cudaError_t launch_tile_keys(const uint32_t *perm, int64_t E, const uint32_t *tid_of, uint32_t *tkey,
                             cudaStream_t s) {
    k_tile_keys<<<blocks(E), kThreads, 0, s>>>(perm, E, tid_of, tkey);
    return cudaGetLastError();
}
cudaError_t launch_group_starts(const uint32_t *vkey, const uint32_t *tkey, int64_t E, uint32_t *flags,
                                cudaStream_t s) {
    k_group_starts<<<blocks(E), kThreads, 0, s>>>(vkey, tkey, E, flags);
    return cudaGetLastError();
}
cudaError_t launch_group_ids(const uint32_t *starts, const uint32_t *excl, int64_t E, uint32_t *gid,
                             cudaStream_t s) {
    k_group_ids<<<blocks(E), kThreads, 0, s>>>(starts, excl, E, gid);
    return cudaGetLastError();
}
cudaError_t launch_tile_major(const uint32_t *tperm, const uint32_t *perm, const uint32_t *gid,
                              const int64_t *tile_E, const uint32_t *tid_of, int64_t E, uint16_t *lidx,
                              uint32_t *ends, uint32_t *tstart, cudaStream_t s) {
    k_tile_major<<<blocks(E), kThreads, 0, s>>>(tperm, perm, gid, tile_E, tid_of, E, lidx, ends, tstart);
    return cudaGetLastError();
}
cudaError_t launch_group_slots(const uint32_t *tperm, const uint32_t *gid, const uint32_t *tstart,
                               const uint32_t *tmi, const int64_t *tile_E, const uint32_t *tid_of, int64_t ntiles,
                               int64_t E, uint32_t *tp2, int64_t *tg_off, cudaStream_t s) {
    k_group_slots<<<blocks(E), kThreads, 0, s>>>(tperm, gid, tstart, tmi, tile_E, tid_of, ntiles, E, tp2, tg_off);
    return cudaGetLastError();
}
cudaError_t launch_seg_groups(const uint32_t *seg_off, int64_t S, const uint32_t *gid, int64_t G, uint32_t *seg_off2,
                              cudaStream_t s) {
    k_seg_groups<<<blocks(S + 1), kThreads, 0, s>>>(seg_off, S, gid, G, seg_off2);
    return cudaGetLastError();
}

}  // namespace mrf
