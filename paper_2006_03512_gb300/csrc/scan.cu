// Device-wide exclusive prefix sums (reduce-then-scan over 4096-item tiles).
// Used for ray offsets (edge counts per pixel -> CSR offsets), the radix-sort
// digit offsets and the voxel-segment numbering.
#include "mrf_internal.cuh"

namespace mrf {
namespace {

using u64 = unsigned long long;

template <typename T>
__device__ __forceinline__ T warp_inclusive_add(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block-wide sum over kThreads threads; also returns the block total.
__device__ __forceinline__ u64 block_exclusive_add(u64 v, u64 &total) {
    __shared__ u64 s_warp[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u64 inc = warp_inclusive_add(v);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    u64 pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        const u64 x = s_warp[w];
        if (w < warp) pre += x;
        tot += x;
    }
    __syncthreads();
    total = tot;
    return pre + inc - v;
}

template <typename In>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const In *__restrict__ in, int64_t n,
                                                          u64 *__restrict__ partials) {
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
    u64 s = 0;
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = t0 + (int64_t)i * kThreads + threadIdx.x;
        if (idx < n) s += (u64)in[idx];
    }
    u64 tot;
    block_exclusive_add(s, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// One CTA scans the tile partials in place (exclusive), chunk by chunk with a
// carried prefix, and stores the grand total at partials[ntiles].
__global__ void __launch_bounds__(kThreads) k_scan_partials(u64 *__restrict__ partials, int64_t ntiles) {
    u64 carry = 0;
    for (int64_t c0 = 0; c0 < ntiles; c0 += kTile) {
        u64 v[kItems];
        u64 s = 0;
        const int64_t b = c0 + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            v[i] = (b + i < ntiles) ? partials[b + i] : 0;
            s += v[i];
        }
        u64 tot;
        u64 pre = block_exclusive_add(s, tot) + carry;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (b + i < ntiles) partials[b + i] = pre;
            pre += v[i];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[ntiles] = carry;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const In *__restrict__ in, Out *__restrict__ out, int64_t n,
                                                        const u64 *__restrict__ partials, int64_t ntiles,
                                                        int64_t base) {
    const int64_t b = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    u64 v[kItems];
    u64 s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        v[i] = (b + i < n) ? (u64)in[b + i] : 0;
        s += v[i];
    }
    u64 tot;
    u64 pre = block_exclusive_add(s, tot) + partials[blockIdx.x] + (u64)base;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (b + i < n) out[b + i] = (Out)pre;
        pre += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (Out)(partials[ntiles] + (u64)base);
}

template <typename Out>
__global__ void k_set_value(Out *p, Out v) { *p = v; }

template <typename In, typename Out>
cudaError_t exclusive_scan(const In *in, Out *out, int64_t n, int64_t base, void *ws, cudaStream_t s) {
    if (n <= 0) {
        k_set_value<Out><<<1, 1, 0, s>>>(out, (Out)base);
        return cudaGetLastError();
    }
    const int64_t ntiles = ceil_div(n, kTile);
    u64 *partials = (u64 *)ws;
    k_tile_reduce<In><<<(unsigned)ntiles, kThreads, 0, s>>>(in, n, partials);
    k_scan_partials<<<1, kThreads, 0, s>>>(partials, ntiles);
    k_tile_scan<In, Out><<<(unsigned)ntiles, kThreads, 0, s>>>(in, out, n, partials, ntiles, base);
    return cudaGetLastError();
}

}  // namespace

size_t scan_workspace_bytes(int64_t n) { return (size_t)(ceil_div(n > 0 ? n : 1, kTile) + 1) * sizeof(u64); }

cudaError_t exclusive_scan_i32_i64(const int32_t *in, int64_t *out, int64_t n, int64_t base, void *ws,
                                   cudaStream_t s) {
    return exclusive_scan<int32_t, int64_t>(in, out, n, base, ws, s);
}

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, void *ws, cudaStream_t s) {
    return exclusive_scan<uint32_t, uint32_t>(in, out, n, 0, ws, s);
}

}  // namespace mrf
