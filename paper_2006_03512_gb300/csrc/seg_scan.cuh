// Segmented sums over a CTA: (partial sum, Kahan compensation, segment ends
// seen) aggregates and their exclusive block-wide scan.  Used by the voxel
// totals and by the ray kernel's per-tile voxel grouping.
#pragma once

#include "mrf_internal.cuh"

namespace mrf {
namespace seg {

template <typename V>
struct SegAgg {
    V s;      // sum since the last segment end (or of everything, if none)
    V cs;     // Kahan compensation of s
    int n;    // segment ends seen
};

template <typename V>
__device__ __forceinline__ void kahan_add(V &s, V &c, V x) {
    const V y = x - c;
    const V t = s + y;
    c = (t - s) - y;
    s = t;
}

template <bool KAHAN, typename V>
__device__ __forceinline__ void acc_add(V &s, V &c, V x) {
    if (KAHAN) kahan_add(s, c, x);
    else s += x;
}

template <typename V>
__device__ __forceinline__ SegAgg<V> seg_op(const SegAgg<V> &a, const SegAgg<V> &b) {  // a precedes b
    if (b.n) return {b.s, b.cs, a.n + b.n};
    return {a.s + (b.s - b.cs) - a.cs, (V)0, a.n};
}

template <typename V>
__device__ __forceinline__ SegAgg<V> shfl_up(const SegAgg<V> &a, int o) {
    return {__shfl_up_sync(0xffffffffu, a.s, o), __shfl_up_sync(0xffffffffu, a.cs, o),
            __shfl_up_sync(0xffffffffu, a.n, o)};
}

template <typename V>
__device__ __forceinline__ SegAgg<V> block_seg_exclusive(SegAgg<V> v, SegAgg<V> *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SegAgg<V> inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const SegAgg<V> y = shfl_up(inc, o);
        if (lane >= o) inc = seg_op(y, inc);
    }
    SegAgg<V> ex = shfl_up(inc, 1);
    if (lane == 0) ex = {(V)0, (V)0, 0};
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    SegAgg<V> pre = {(V)0, (V)0, 0};
    for (int w = 0; w < warp; ++w) pre = seg_op(pre, s_w[w]);
    return seg_op(pre, ex);
}


}  // namespace seg
}  // namespace mrf
