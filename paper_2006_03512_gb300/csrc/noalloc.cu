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

// The device address of g_reduce_scratch is looked up once per device and
// context, with that device current, and kept with the context's unique id: a
// device reset (or another context made current on the same device) gives a
// new id, and the address is looked up again, since the library's module may
// then be loaded at another address.
using CtxGetCurrent = int (*)(void **);
using CtxGetId = int (*)(void *, unsigned long long *);
struct Cached {
    unsigned long long ctx_id = 0;
    void *addr = nullptr;
};
std::mutex g_lock;
Cached g_cache[128];
CtxGetCurrent g_get_ctx = nullptr;
CtxGetId g_get_id = nullptr;

// The unique id of the calling thread's current context (0 if none is current
// yet, or if the driver cannot report one).
unsigned long long current_ctx_id() {
    if (!g_get_ctx || !g_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return 0;
        g_get_ctx = reinterpret_cast<CtxGetCurrent>(f1);
        g_get_id = reinterpret_cast<CtxGetId>(f2);
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_get_ctx(&ctx) != 0 || !ctx || g_get_id(ctx, &id) != 0) return 0;
    return id;
}

// The device address of the scratch array for the current device and context.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MRF_ECUDA;
    if (dev < 0 || dev >= 128) return MRF_ERANGE;
    std::lock_guard<std::mutex> guard(g_lock);
    unsigned long long id = current_ctx_id();
    Cached &c = g_cache[dev];
    if (id == 0 || c.ctx_id != id || !c.addr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess || !p) return MRF_ECUDA;
        id = current_ctx_id();   // the lookup makes the runtime's context current if none was
        c.addr = p;
        c.ctx_id = id;           // 0: no id available, looked up again on the next call
    }
    *out = c.addr;
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
