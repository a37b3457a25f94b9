// Voxel totals without any allocation: the same kernels as mrf_voxel_reduce,
// with their scratch (per-tile plans and partial sums) in a statically sized
// device array that the library defines once.
//
// This is for callers that cannot allocate device memory when they call in:
// a mapping loop that runs under a fixed, preallocated memory budget (for
// instance on a robot where an allocation failure mid-run is not acceptable),
// or code that runs inside a memory allocator's own callbacks and must not
// re-enter it.  They pass their inputs and outputs; the library provides the
// scratch.
#include <mutex>

#include "mrf_internal.cuh"
#include "mrfmap.h"

namespace {

using namespace mrf;

constexpr int64_t kMaxEdges = MRF_NOALLOC_MAX_EDGES;
constexpr int64_t kMaxTiles = kMaxEdges / kTile;
// plan (two u32 per tile), head partials (f32), tail partials (f32), tail
// segment ids (u32): 20 bytes per 4096-edge tile, 1.25 MiB in all
constexpr size_t kScratchBytes = (size_t)kMaxTiles * (8 + 4 + 4 + 4);

// Lives on every device that loads the library until the process exits.  Host
// code must not use the symbol as an address; it asks the runtime for the
// device address below.
static __device__ __align__(256) unsigned char g_reduce_scratch[kScratchBytes];

std::mutex g_lock;
void *g_addr[128] = {};  // device address of g_reduce_scratch, per device ordinal

// Looks up (once per device, with that device current) the device address of
// the scratch array.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MRF_ECUDA;
    if (dev < 0 || dev >= 128) return MRF_ERANGE;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess || !p) return MRF_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MRF_OK;
}

}  // namespace

extern "C" int mrf_voxel_reduce_noalloc(const uint32_t *perm_dev, const uint32_t *seg_off_dev,
                                        const uint32_t *seg_vox_dev, int64_t n_seg, int64_t n_edges,
                                        const float *lam_dev, float logit_prior, float *T_dev, void *stream) {
    if (n_edges < 0 || n_seg < 0) return MRF_EINVAL;
    if (n_edges > kMaxEdges) return MRF_ERANGE;
    if (n_edges == 0) return MRF_OK;
    if (n_seg == 0 || !perm_dev || !seg_off_dev || !seg_vox_dev || !lam_dev || !T_dev) return MRF_EINVAL;
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != MRF_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nt = ceil_div(n_edges, kTile);
    // every scratch word a call reads is written earlier in the same call, so
    // nothing has to be cleared between calls
    char *w = (char *)ws;
    uint32_t *plan = (uint32_t *)w;
    float *head = (float *)(w + kMaxTiles * 8);
    float *tail = (float *)(w + kMaxTiles * 12);
    uint32_t *tseg = (uint32_t *)(w + kMaxTiles * 16);
    if (launch_reduce_plan(seg_off_dev, n_seg, n_edges, plan, nt, s) != cudaSuccess) return MRF_ECUDA;
    if (launch_voxel_reduce_f32(perm_dev, seg_off_dev, seg_vox_dev, plan, nt, lam_dev, T_dev, logit_prior, n_edges,
                                head, tail, tseg, s) != cudaSuccess)
        return MRF_ECUDA;
    return MRF_OK;
}
