// Voxel-sorted transpose of the ray->voxel edges: a stable LSD radix sort of
// (voxel index, edge id) pairs, 8 bits per pass, followed by the list of
// non-empty voxels (segments) with their start offsets.
//
// The paper accumulates ray contributions into voxels with atomics
// (Section IV-A); atomics make the summation order, and so the rounding,
// depend on scheduling.  Sorting once per build instead gives every voxel a
// fixed, edge-id-ordered list, so the per-voxel sums are bitwise reproducible.
//
// Each pass is count -> exclusive scan of the (digit, tile) table -> stable
// scatter.  Stability inside a 4096-key tile comes from warp-ordered ranking:
// warp w owns keys [w*512, (w+1)*512) of the tile, walks them in order 32 at a
// time, and ranks equal digits with __match_any_sync; per-warp digit counts are
// then prefixed across warps in warp order.  The ranked tile is reordered in
// shared memory before it is written, so the global stores of a digit's run
// are consecutive.
#include "mrf_internal.cuh"

namespace mrf {
namespace {

constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;
constexpr int kWarps = kThreads / 32;
constexpr int kKeysPerWarp = kTile / kWarps;  // 512
constexpr int kRounds = kKeysPerWarp / 32;    // 16

__global__ void __launch_bounds__(kThreads) k_rs_count(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                       uint32_t *__restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t cnt[kDigits];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = t0 + (int64_t)i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix of v over the CTA's threads (thread order); s_w holds
// kWarps words.  Every thread calls it; it contains one barrier.
__device__ __forceinline__ uint32_t cta_exclusive(uint32_t v, uint32_t *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    uint32_t pre = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
        if (w < warp) pre += s_w[w];
    return pre + inc - v;
}

// One stable scatter pass.  The tile's keys are ranked (warp order, then
// __match_any_sync within a warp), placed in shared memory in their sorted
// order within the tile, and written out from there in that order: a digit's
// run of the tile goes to consecutive global positions, so consecutive threads
// store to consecutive addresses.  The result is the same as ranking straight
// into global memory.
__global__ void __launch_bounds__(kThreads, 2) k_rs_scatter(const uint32_t *__restrict__ keys_in,
                                                         const uint32_t *__restrict__ vals_in,
                                                         uint32_t *__restrict__ keys_out,
                                                         uint32_t *__restrict__ vals_out, int64_t n, int shift,
                                                         const uint32_t *__restrict__ offs, int64_t ntiles) {
    __shared__ uint32_t wcnt[kWarps][kDigits];
    __shared__ uint32_t dbase[kDigits];   // global first position of the tile's keys of each digit
    __shared__ uint32_t dloc[kDigits];    // first position of each digit in the tile's sorted order
    __shared__ uint32_t s_w[kWarps];
    __shared__ uint32_t skey[kTile], sval[kTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
    dbase[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tbase = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = tbase + (int64_t)warp * kKeysPerWarp;
    uint32_t key[kRounds], val[kRounds], dr[kRounds];   // dr: rank << 9 | digit (kDigits = invalid)
    // every load first, so that their latencies overlap
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? keys_in[idx] : 0u;
        val[r] = valid ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        const uint32_t k = key[r];
        const int d = valid ? (int)((k >> shift) & (kDigits - 1)) : kDigits;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = __popc(peers & lt_mask);
        uint32_t base = 0;
        if (valid) base = wcnt[warp][d];
        __syncwarp();
        if (valid && before == 0) wcnt[warp][d] = base + __popc(peers);
        __syncwarp();
        dr[r] = ((base + before) << 9) | (uint32_t)d;
    }
    __syncthreads();
    uint32_t total;
    {   // per digit, exclusive prefix over warps (warp order = key order), and the digit's tile count
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
        total = run;
    }
    dloc[threadIdx.x] = cta_exclusive(total, s_w);   // its barrier also publishes wcnt
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int d = (int)(dr[r] & 511u);
        if (d < kDigits) {
            const uint32_t lp = dloc[d] + wcnt[warp][d] + (dr[r] >> 9);
            skey[lp] = key[r];
            sval[lp] = val[r];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - tbase < kTile ? n - tbase : kTile);
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
        const uint32_t k = skey[i];
        const int d = (int)((k >> shift) & (kDigits - 1));
        const uint32_t g = dbase[d] + (uint32_t)i - dloc[d];
        keys_out[g] = k;
        vals_out[g] = sval[i];
    }
}

__global__ void __launch_bounds__(kThreads) k_seg_heads(const uint32_t *__restrict__ k, int64_t n,
                                                        uint32_t *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) flags[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void __launch_bounds__(kThreads) k_seg_emit(const uint32_t *__restrict__ k,
                                                       const uint32_t *__restrict__ head_idx, int64_t n,
                                                       uint32_t *__restrict__ seg_off, uint32_t *__restrict__ seg_vox) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || k[i] != k[i - 1]) {
        const uint32_t s = head_idx[i];
        seg_off[s] = (uint32_t)i;
        seg_vox[s] = k[i];
    }
    if (i == n - 1) seg_off[head_idx[n]] = (uint32_t)n;
}

}  // namespace

size_t sort_workspace_bytes(int64_t n) {
    const int64_t ntiles = ceil_div(n > 0 ? n : 1, kTile);
    const int64_t hist = (int64_t)kDigits * ntiles;
    // digit table, its scan (hist + 1 entries) and the scan's own workspace
    return (size_t)(2 * hist + 1) * sizeof(uint32_t) + 64 + scan_workspace_bytes(hist);
}

cudaError_t radix_sort_edges(const uint32_t *keys_in, int key_bits, int64_t n, uint32_t *keys_a, uint32_t *keys_b,
                             uint32_t *vals_tmp, uint32_t *vals_out, uint32_t **keys_sorted, void *ws,
                             cudaStream_t s, int64_t *n_launches) {
    const int passes = key_bits <= 0 ? 1 : (key_bits + kRadixBits - 1) / kRadixBits;
    const int64_t ntiles = ceil_div(n, kTile);
    const int64_t hsize = (int64_t)kDigits * ntiles;
    uint32_t *hist = (uint32_t *)ws;
    uint32_t *offs = hist + hsize;
    void *scan_ws = (void *)(((uintptr_t)(offs + hsize + 1) + 15) & ~(uintptr_t)15);
    const uint32_t *kin = keys_in;
    const uint32_t *vin = nullptr;  // identity: edge ids
    for (int p = 0; p < passes; ++p) {
        // the last pass lands in vals_out / keys_a
        const bool to_final = ((passes - 1 - p) % 2) == 0;
        uint32_t *kout = to_final ? keys_a : keys_b;
        uint32_t *vout = to_final ? vals_out : vals_tmp;
        const int shift = p * kRadixBits;
        k_rs_count<<<(unsigned)ntiles, kThreads, 0, s>>>(kin, n, shift, hist, ntiles);
        cudaError_t e = exclusive_scan_u32(hist, offs, hsize, scan_ws, s);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(kin, vin, kout, vout, n, shift, offs, ntiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (n_launches) *n_launches += 5;
        kin = kout;
        vin = vout;
    }
    *keys_sorted = keys_a;
    return cudaSuccess;
}

cudaError_t segment_heads(const uint32_t *sorted_keys, int64_t n, uint32_t *flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_seg_heads<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(sorted_keys, n, flags);
    return cudaGetLastError();
}

cudaError_t segment_emit(const uint32_t *sorted_keys, const uint32_t *head_idx, int64_t n, uint32_t *seg_off,
                         uint32_t *seg_vox, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_seg_emit<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(sorted_keys, head_idx, n, seg_off, seg_vox);
    return cudaGetLastError();
}

}  // namespace mrf
