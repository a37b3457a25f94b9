// C ABI of the library (declared in include/mrfmap.h): context, memory, frame
// ingest, transpose build, the BP iteration loop, exports and profiling.
#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <utility>
#include <vector>

#include "mrf_internal.cuh"

#include "mrfmap.h"

using namespace mrf;

namespace {

// Stream-ordered device buffer owned by a context.
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct EventPair {
    cudaEvent_t a, b;
    int kind;
};

enum Kind { K_RAY = 0, K_RED = 1, K_OTHER = 2, K_BUILD = 3, K_TRAV = 4 };

}  // namespace

struct mrf_ctx {
    mrf_grid g;                    // scene 0 (the only scene of an mrf_create context)
    float prior;
    mrf_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int64_t V = 0;                 // nx * ny * nz
    int64_t Vk = 0;                // internal key space (whole 8^3 bricks), all scenes
    struct Scene {
        mrf_grid g;
        GridMap gm;
        int64_t V, key_base, lin_base;   // voxels; first key; first linear index in the marginals
    };
    std::vector<Scene> scenes;
    // kernel plan chosen by the caller (mrf_set_plan); 0 / -1: the library's choice
    int plan_items = 0, plan_threads = 0, plan_groups = -1;
    // CUDA graph of a whole mrf_infer (mrf_infer_graph)
    cudaGraphExec_t graph = nullptr;
    int32_t graph_iters = -1;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    bool capturing = false;
    int64_t graph_launches = 0;    // kernels one replay runs
    GridMap gm;

    // frames and edges
    int64_t R = 0, E = 0, cap_R = 0, cap_E = 0;
    int32_t max_len = 0;
    int n_frames = 0;
    double nu_bg = -1.0;   // all-empty likelihood, resolved at the first frame
    float nu_floor = FLT_MAX;   // smallest likelihood floor (w / d_hi) of the frames' tables
    double nu_max = 0.0;        // bound on every likelihood: (1 - w) / (sqrt(2 pi) sigma_min) + w / d_hi
    // held-out rays (mrf_add_heldout) and the gradient's buffers (mrf_grad)
    Buf h_ray_off, h_Zr, h_vox, h_dmid;
    int64_t hR = 0, hE = 0, h_capR = 0, h_capE = 0;
    Buf gr_ck_lam, gr_ck_T, gr_gT, gr_glam, gr_gL, gr_gLn, gr_gnu, gr_sP, gr_sA, gr_sB, gr_sg, gr_gbg, gr_head,
        gr_tail, gr_tseg, gr_part, gr_hQ, gr_hnu, gr_hgp, gr_hgnu, gr_hloss, gr_hgbg, gr_hperm, gr_hso, gr_hsv,
        gr_hplan;
    Buf ray_off, Zr, vox, dmid, nu, nu64;
    // the accuracy metric's per-frame scratch (mrf_accuracy)
    Buf ac_ray_off, ac_Z, ac_vox, ac_tin, ac_tout, ac_cnt;
    // the implementation variants: per-edge length weights, each frame's first
    // edge, and the (keyframe, voxel) pairs over the voxel-major order
    Buf wlen, pair_off, frame_E_dev, pair_pid, pair_ident, pair_sum, pair_plan, pair_head, pair_tail, pair_tseg;
    std::vector<int64_t> frame_E;
    int64_t n_pairs = 0, n_pair_tiles = 0;
    // rays longer than opt.long_ray_f64 edges (FP64 accumulations): ids, offsets
    // into the compact message and scratch arrays
    Buf lr_ids, lr_off, lr_out, lr_scr;
    int64_t n_long = 0;
    // transpose
    bool dirty = true;
    bool have_perm = false;   // the per-edge transpose (perm, seg_off, red_plan) is built
    int64_t n_seg = 0;
    Buf perm, seg_off, seg_vox;
    // messages
    Buf lam, T, lam64, T64, bscr64;
    // plans and scratch
    int kt = 0;
    int64_t n_ray_tiles = 0, n_red_tiles = 0;
    Buf ray_plan, red_plan, head_part, tail_part, tail_seg;
    Buf tile_E, ray_starts;        // pipelined ray kernel: tile edge bounds, ray-start bitmap
    // pre-aggregation: per-(tile, voxel) groups
    bool use_groups = false;
    int pipe_nt = kThreads;        // threads per CTA of the pipelined ray kernel
    int64_t n_groups = 0, n_red2 = 0;
    Buf g_lidx, g_ends, g_gid, g_key, g_tg_off, g_tp2, g_seg_off2, g_partial, g_plan, g_head, g_tail, g_tseg;
    bool use_pipe = false;
    int n_sm = 0;
    Buf err_dev;                   // device-side error word (bounded waits)
    int64_t fail_alloc_at = 0;     // injected failure: the n-th device allocation from now (0: off)
    int64_t alloc_count = 0;
    // staging
    Buf counts, maxlen_dev, scan_ws, depth_stage;
    Buf rsetup;                    // per pixel of the frame being walked: its ray set-up
    int64_t *h_pinned = nullptr;  // 4 int64 of pinned host memory for read-backs
    // status
    int sticky = MRF_OK;
    std::string err;
    // profiling
    bool profiling = false;
    std::vector<EventPair> events;
    std::vector<cudaEvent_t> event_pool;
    int64_t launches = 0;
};

namespace {

constexpr int64_t kPad = 8192;  // elements of slack after per-edge arrays (vector tails)

int fail(mrf_ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(mrf_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        if (c->sticky == MRF_OK) {
            c->sticky = code;
            c->err = buf;
        }
    }
    return code;
}

#define CUDA_TRY(c, expr)                                                                                   \
    do {                                                                                                    \
        cudaError_t _e = (expr);                                                                            \
        if (_e != cudaSuccess)                                                                              \
            return fail((c), _e == cudaErrorMemoryAllocation ? MRF_ENOMEM : MRF_ECUDA, "%s: %s (%s:%d)", #expr, \
                        cudaGetErrorString(_e), __FILE__, __LINE__);                                        \
    } while (0)

#define TRY(expr)                    \
    do {                             \
        int _r = (expr);             \
        if (_r != MRF_OK) return _r; \
    } while (0)

int ensure(mrf_ctx *c, Buf &b, size_t bytes, bool keep) {
    if (bytes <= b.bytes) return MRF_OK;
    if (c->fail_alloc_at > 0 && ++c->alloc_count == c->fail_alloc_at) {
        c->fail_alloc_at = 0;
        return fail(c, MRF_ENOMEM, "device allocation of %zu bytes failed: injected", bytes);
    }
    void *np = nullptr;
    cudaError_t e = cudaMallocAsync(&np, bytes, c->stream);
    if (e != cudaSuccess) {
        // what the pool holds of freed buffers goes back to the device; once more
        cudaGetLastError();
        cudaStreamSynchronize(c->stream);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocAsync(&np, bytes, c->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MRF_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    if (keep && b.p && b.bytes) CUDA_TRY(c, cudaMemcpyAsync(np, b.p, b.bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (b.p) CUDA_TRY(c, cudaFreeAsync(b.p, c->stream));
    b.p = np;
    b.bytes = bytes;
    return MRF_OK;
}

void release(mrf_ctx *c, Buf &b) {
    if (b.p) cudaFreeAsync(b.p, c->stream);
    b.p = nullptr;
    b.bytes = 0;
}

// A function's temporary device buffer: released on every way out, including
// the early returns of a failed step.
struct Scratch : Buf {
    mrf_ctx *c;
    explicit Scratch(mrf_ctx *c_) : c(c_) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch() { release(c, *this); }
};

template <typename T>
T *ptr(const Buf &b) {
    return reinterpret_cast<T *>(b.p);
}

cudaEvent_t take_event(mrf_ctx *c) {
    cudaEvent_t e;
    if (!c->event_pool.empty()) {
        e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets a group of launches of one kernel class with events when profiling.
struct Prof {
    mrf_ctx *c;
    int kind;
    cudaEvent_t a = nullptr;
    Prof(mrf_ctx *c_, int k) : c(c_), kind(k) {
        if (c->profiling && !c->capturing && (a = take_event(c))) cudaEventRecord(a, c->stream);
    }
    ~Prof() {
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) return;
        cudaEventRecord(b, c->stream);
        c->events.push_back({a, b, kind});
    }
};

int check_ctx(mrf_ctx *c) {
    if (!c) return MRF_EINVAL;
    if (c->sticky != MRF_OK) return c->sticky;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, MRF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return MRF_OK;
}

int key_bits(int64_t V) {
    int b = 0;
    while (b < 32 && ((V - 1) >> b) > 0) ++b;
    return b < 1 ? 1 : b;
}

float logitf_(double p) { return (float)(log(p) - log1p(-p)); }

// ------------------------------------------------------------------ build
// Per-(tile, voxel) groups for the pre-aggregating ray kernel (see group.cu).
// Each tile's edges are grouped by voxel in shared memory, which gives the
// tile-major order (window indices, group ends, group counts); the groups'
// voxel keys are then sorted once (stable, so tile order within a voxel) for
// the voxel totals.  ka, kb, vt: (E+1)-entry scratch; ws: the transpose's sort
// workspace (sized for E >= G).
int build_groups(mrf_ctx *c, uint32_t *ka, uint32_t *kb, uint32_t *vt, Buf &ws) {
    const int64_t E = c->E, nt = c->n_ray_tiles;
    const int64_t *tE = ptr<int64_t>(c->tile_E);
    const int cap = c->pipe_nt * c->kt;
    const int64_t words = (E + kPad) / 32 + 2;
    TRY(ensure(c, c->g_lidx, (size_t)(E + kPad) * 2, false));
    // window indices past the last edge are read (unmasked) by the ray kernel's
    // epilogue: keep them in range
    CUDA_TRY(c, cudaMemsetAsync(ptr<uint16_t>(c->g_lidx) + E, 0, (size_t)kPad * 2, c->stream));
    TRY(ensure(c, c->g_ends, (size_t)words * 4, false));
    TRY(ensure(c, c->g_gid, (size_t)(E + kPad) * 2, false));
    // group indices past the last edge are read (and masked) by the ray kernel: keep them in range
    CUDA_TRY(c, cudaMemsetAsync(ptr<uint16_t>(c->g_gid) + E, 0, (size_t)kPad * 2, c->stream));
    TRY(ensure(c, c->g_tg_off, (size_t)(nt + 1) * 8, false));
    CUDA_TRY(c, cudaMemsetAsync(c->g_ends.p, 0, (size_t)words * 4, c->stream));
    // per tile: sorted window indices, group ends, group counts (into vt)
    // (each tile's group keys go to ka at the tile's first edge, for launch_group_keys)
    CUDA_TRY(c, launch_tile_sort(cap, tE, nt, ptr<uint32_t>(c->ray_starts), ptr<uint32_t>(c->vox), ptr<uint16_t>(c->g_lidx),
                                 ptr<uint32_t>(c->g_ends), ptr<uint16_t>(c->g_gid), reinterpret_cast<int32_t *>(vt), ka,
                                 c->stream));
    CUDA_TRY(c, exclusive_scan_i32_i64(reinterpret_cast<const int32_t *>(vt), ptr<int64_t>(c->g_tg_off), nt, 0, ws.p,
                                       c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<int64_t>(c->g_tg_off) + nt, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t G = c->h_pinned[0];
    c->n_groups = G;
    // group keys by slot (kept: the ray kernel gathers one voxel total per
    // group), then their stable voxel order: tp2[voxel-order index] = slot
    TRY(ensure(c, c->g_key, (size_t)(G + kPad) * 4, false));
    CUDA_TRY(c, launch_group_keys(tE, nt, ptr<int64_t>(c->g_tg_off), ka, ptr<uint32_t>(c->g_key), c->stream));
    uint32_t *gkey = ptr<uint32_t>(c->g_key);
    TRY(ensure(c, c->g_tp2, (size_t)(G + kPad) * 4, false));
    uint32_t *gsorted = nullptr;
    CUDA_TRY(c, radix_sort_edges(gkey, key_bits(c->Vk), G, ka, kb, vt, ptr<uint32_t>(c->g_tp2), &gsorted,
                                 ws.p, c->stream, &c->launches));
    // groups per voxel: runs of the sorted keys, one per non-empty voxel (the
    // segments: seg_vox lists the non-empty voxels' keys in order)
    uint32_t *gflags = gsorted == ka ? kb : ka;
    CUDA_TRY(c, segment_heads(gsorted, G, gflags, c->stream));
    CUDA_TRY(c, exclusive_scan_u32(gflags, vt, G, ws.p, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, vt + G, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t S = (int64_t)(*(uint32_t *)c->h_pinned);
    c->n_seg = S;
    TRY(ensure(c, c->g_seg_off2, (size_t)(S + 1) * 4, false));
    TRY(ensure(c, c->seg_vox, (size_t)(S > 0 ? S : 1) * 4, false));
    CUDA_TRY(c, segment_emit(gsorted, vt, G, ptr<uint32_t>(c->g_seg_off2), ptr<uint32_t>(c->seg_vox), c->stream));
    // voxel totals over groups
    c->n_red2 = ceil_div(G, kTile);
    TRY(ensure(c, c->g_partial, (size_t)(G + kPad) * 4, false));
    TRY(ensure(c, c->g_plan, (size_t)c->n_red2 * 8, false));
    TRY(ensure(c, c->g_head, (size_t)c->n_red2 * 4, false));
    TRY(ensure(c, c->g_tail, (size_t)c->n_red2 * 4, false));
    TRY(ensure(c, c->g_tseg, (size_t)c->n_red2 * 4, false));
    CUDA_TRY(c, launch_reduce_plan(ptr<uint32_t>(c->g_seg_off2), S, G, ptr<uint32_t>(c->g_plan), c->n_red2,
                                   c->stream));
    c->launches += 8;
    return MRF_OK;
}

// (keyframe, voxel) pairs for MRF_VAR_KEYFRAME_AVG: runs of equal (voxel,
// frame) in the voxel-major edge order, as offsets into it.
int build_pairs(mrf_ctx *c) {
    const int64_t E = c->E;
    const int32_t nf = (int32_t)c->frame_E.size();
    Scratch flags(c), pos(c), ws(c);
    TRY(ensure(c, c->frame_E_dev, (size_t)nf * 8, false));
    TRY(ensure(c, flags, (size_t)E * 4, false));
    TRY(ensure(c, pos, (size_t)(E + 1) * 8, false));
    TRY(ensure(c, ws, scan_workspace_bytes(E), false));
    CUDA_TRY(c, cudaMemcpyAsync(c->frame_E_dev.p, c->frame_E.data(), (size_t)nf * 8, cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, launch_pair_flags(ptr<uint32_t>(c->perm), ptr<uint32_t>(c->vox), E, ptr<int64_t>(c->frame_E_dev), nf,
                                  ptr<int32_t>(flags), c->stream));
    CUDA_TRY(c, exclusive_scan_i32_i64(ptr<int32_t>(flags), ptr<int64_t>(pos), E, 0, ws.p, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<int64_t>(pos) + E, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->n_pairs = c->h_pinned[0];
    TRY(ensure(c, c->pair_off, (size_t)(c->n_pairs + 1) * 4, false));
    TRY(ensure(c, c->pair_ident, (size_t)(c->n_pairs + 1) * 4, false));
    TRY(ensure(c, c->pair_sum, (size_t)(c->n_pairs + 1) * 4, false));
    TRY(ensure(c, c->pair_pid, (size_t)(E + 1) * 4, false));
    CUDA_TRY(c, launch_pair_starts(ptr<int32_t>(flags), ptr<int64_t>(pos), E, ptr<uint32_t>(c->pair_off),
                                   ptr<uint32_t>(c->pair_pid), ptr<uint32_t>(c->pair_ident), c->stream));
    // the pair sums reuse the voxel totals' segmented reduction over pairs
    c->n_pair_tiles = ceil_div(E, kTile);
    TRY(ensure(c, c->pair_plan, (size_t)c->n_pair_tiles * 8, false));
    TRY(ensure(c, c->pair_head, (size_t)c->n_pair_tiles * 4, false));
    TRY(ensure(c, c->pair_tail, (size_t)c->n_pair_tiles * 4, false));
    TRY(ensure(c, c->pair_tseg, (size_t)c->n_pair_tiles * 4, false));
    CUDA_TRY(c, launch_reduce_plan(ptr<uint32_t>(c->pair_off), c->n_pairs, E, ptr<uint32_t>(c->pair_plan),
                                   c->n_pair_tiles, c->stream));
    c->launches += 4;
    release(c, flags);
    release(c, pos);
    release(c, ws);
    return MRF_OK;
}

// The edge-level voxel transpose: the stable radix sort of (voxel, edge id)
// into perm, the non-empty voxels (segments) and the per-edge reduction plan.
// The grouped FP32 path does not need it (its voxel totals run over groups,
// whose own sort yields the segments); it is built when a path or an export
// asks for it.
int build_edge_transpose(mrf_ctx *c) {
    const int64_t E = c->E;
    Scratch ka(c), kb(c), vt(c), ws(c);
    TRY(ensure(c, c->perm, (size_t)(E + kPad) * 4, false));
    TRY(ensure(c, ka, (size_t)(E + 1) * 4, false));
    TRY(ensure(c, kb, (size_t)(E + 1) * 4, false));
    TRY(ensure(c, vt, (size_t)(E + 1) * 4, false));
    size_t wsb = sort_workspace_bytes(E);
    const size_t swb = scan_workspace_bytes(E);
    if (swb > wsb) wsb = swb;
    TRY(ensure(c, ws, wsb, false));
    uint32_t *sorted = nullptr;
    CUDA_TRY(c, radix_sort_edges(ptr<uint32_t>(c->vox), key_bits(c->Vk), E, ptr<uint32_t>(ka), ptr<uint32_t>(kb),
                                 ptr<uint32_t>(vt), ptr<uint32_t>(c->perm), &sorted, ws.p, c->stream, &c->launches));
    // segments = non-empty voxels
    uint32_t *flags = sorted == ptr<uint32_t>(ka) ? ptr<uint32_t>(kb) : ptr<uint32_t>(ka);
    CUDA_TRY(c, segment_heads(sorted, E, flags, c->stream));
    CUDA_TRY(c, exclusive_scan_u32(flags, ptr<uint32_t>(vt), E, ws.p, c->stream));
    c->launches += 4;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<uint32_t>(vt) + E, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t S = (int64_t)(*(uint32_t *)c->h_pinned);
    if (c->use_groups && S != c->n_seg) return fail(c, MRF_ECUDA, "edge and group transposes disagree");
    c->n_seg = S;
    TRY(ensure(c, c->seg_off, (size_t)(S + 1) * 4, false));
    TRY(ensure(c, c->seg_vox, (size_t)(S > 0 ? S : 1) * 4, false));
    CUDA_TRY(c, segment_emit(sorted, ptr<uint32_t>(vt), E, ptr<uint32_t>(c->seg_off), ptr<uint32_t>(c->seg_vox),
                             c->stream));
    c->launches += 1;
    release(c, ka);
    release(c, kb);
    release(c, vt);
    release(c, ws);
    // voxel-reduction tiles over edges
    c->n_red_tiles = ceil_div(E, kTile);
    TRY(ensure(c, c->red_plan, (size_t)c->n_red_tiles * 8, false));
    TRY(ensure(c, c->tail_seg, (size_t)c->n_red_tiles * 4, false));
    const size_t vb = c->opt.precision == MRF_PREC_F64 ? 8 : 4;
    TRY(ensure(c, c->head_part, (size_t)c->n_red_tiles * vb, false));
    TRY(ensure(c, c->tail_part, (size_t)c->n_red_tiles * vb, false));
    CUDA_TRY(c, launch_reduce_plan(ptr<uint32_t>(c->seg_off), S, E, ptr<uint32_t>(c->red_plan), c->n_red_tiles,
                                   c->stream));
    c->launches += 2;
    c->have_perm = true;
    if (c->opt.debug_checks) {
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        std::vector<uint32_t> so((size_t)S + 1);
        CUDA_TRY(c, cudaMemcpy(so.data(), c->seg_off.p, so.size() * 4, cudaMemcpyDeviceToHost));
        if (so[0] != 0 || (int64_t)so[S] != E) return fail(c, MRF_ECUDA, "segment offsets do not span the edges");
        for (int64_t s = 0; s < S; ++s)
            if (so[s + 1] <= so[s]) return fail(c, MRF_ECUDA, "segment %lld is empty", (long long)s);
    }
    return MRF_OK;
}

// The pool keeps freed memory (see mrf_create), so the next build reuses the
// sort's temporaries without mapping them again (a quarter of a rebuild's
// time on the 2.6e9-edge room).  It gives them back to the device when less
// than a quarter of the device is free, when an allocation fails (ensure) and
// when a context is destroyed.
int trim_pool(mrf_ctx *c) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr >= tot / 4) return MRF_OK;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    return MRF_OK;
}

int build_transpose(mrf_ctx *c) {
    const int64_t E = c->E;
    Prof prof(c, K_BUILD);
    c->n_seg = 0;
    c->n_ray_tiles = 0;
    c->use_groups = false;
    c->have_perm = false;
    if (c->graph) {   // its kernels point at the buffers this transpose build may replace
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        c->graph_iters = -1;
    }
    c->n_groups = 0;
    c->n_red_tiles = 0;
    if (E == 0) {
        c->dirty = false;
        return MRF_OK;
    }
    // ray-message tiles
    c->kt = ray_tile_items(c->max_len);
    const bool planned = c->plan_items || c->plan_threads || c->plan_groups >= 0;   // mrf_set_plan
    if (const char *env = planned ? nullptr : getenv("MRF_RAY_ITEMS")) {
        const int v = atoi(env);
        if ((v == 8 || v == 16 || v == 32) && ray_tile_window(v, c->max_len) >= 1) c->kt = v;
    }
    if (c->plan_items >= 8 && ray_tile_window(c->plan_items, c->max_len) >= 1) c->kt = c->plan_items;
    // 512 threads of 4 edges: the pipelined kernel only, on 2048-edge tiles
    const bool pipe4 = c->plan_items == 4 && c->plan_threads == 512 && c->max_len + 8 <= 512 * 4;
    if (c->kt == 0) return fail(c, MRF_ERANGE, "ray of %d edges exceeds the ray kernel's capacity", c->max_len);
    const int64_t window = ray_tile_window(c->kt, c->max_len);
    c->n_ray_tiles = ceil_div(E, window);
    TRY(ensure(c, c->ray_plan, (size_t)(c->n_ray_tiles + 1) * 4, false));
    CUDA_TRY(c, launch_ray_plan(ptr<int64_t>(c->ray_off), c->R, E, window, ptr<uint32_t>(c->ray_plan),
                                c->n_ray_tiles, c->stream));
    // the pipelined kernel: 256 threads, or 128 threads of 16 edges (the same
    // 2048-edge tiles)
    c->pipe_nt = kThreads;
    if (const char *env = planned ? nullptr : getenv("MRF_PIPE_THREADS")) {
        const int v = atoi(env);
        if (v == 128 && c->kt == 16) c->pipe_nt = 128;
    }
    if (c->plan_threads > 0 && ray_pipe_supported(c->kt, c->plan_threads)) c->pipe_nt = c->plan_threads;
    if (pipe4) {
        c->kt = 4;
        c->pipe_nt = 512;
    }
    c->use_pipe = ray_pipe_supported(c->kt, c->pipe_nt) && c->plan_threads >= 0 &&
                  !(c->opt.variants & MRF_VAR_LENGTH_WEIGHT) && c->opt.precision != MRF_PREC_F32_LOG;
    if (const char *env = planned ? nullptr : getenv("MRF_RAY_PIPE")) c->use_pipe = c->use_pipe && atoi(env) != 0;
    if (c->use_pipe) {
        // whole rays packed greedily into tiles of at most (threads * KT) edges
        // (from an edge offset rounded down to 8), in independent chunks of rays
        const int64_t cap = (int64_t)c->pipe_nt * c->kt;
        const int64_t nch = tile_pack_chunks(c->R);
        Scratch cnt(c), off(c), ws(c);
        TRY(ensure(c, cnt, (size_t)nch * 4, false));
        TRY(ensure(c, off, (size_t)(nch + 1) * 8, false));
        TRY(ensure(c, ws, scan_workspace_bytes(nch), false));
        CUDA_TRY(c, launch_tile_pack(ptr<int64_t>(c->ray_off), c->R, cap, ptr<int32_t>(cnt), nullptr, nullptr,
                                     c->stream));
        CUDA_TRY(c, exclusive_scan_i32_i64(ptr<int32_t>(cnt), ptr<int64_t>(off), nch, 0, ws.p, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<int64_t>(off) + nch, 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        const int64_t ntiles = c->h_pinned[0];
        c->n_ray_tiles = ntiles;
        const int64_t words = (E + kPad) / 32 + 2;
        TRY(ensure(c, c->tile_E, (size_t)(ntiles + 1) * 8, false));
        TRY(ensure(c, c->ray_starts, (size_t)words * 4, false));
        CUDA_TRY(c, launch_tile_pack(ptr<int64_t>(c->ray_off), c->R, cap, nullptr, ptr<int64_t>(off),
                                     ptr<int64_t>(c->tile_E), c->stream));
        c->h_pinned[1] = E;
        CUDA_TRY(c, cudaMemcpyAsync(ptr<int64_t>(c->tile_E) + ntiles, c->h_pinned + 1, 8, cudaMemcpyHostToDevice,
                                    c->stream));
        CUDA_TRY(c, launch_ray_pipe_plan(ptr<int64_t>(c->ray_off), c->R, nullptr, 0, nullptr,
                                         ptr<uint32_t>(c->ray_starts), words, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the scratch goes out of scope
        c->launches += 6;
    }
    c->use_groups = c->use_pipe && c->opt.precision != MRF_PREC_F64 && c->opt.long_ray_f64 == 0;
    if (const char *env = planned ? nullptr : getenv("MRF_GROUPS")) c->use_groups = c->use_groups && atoi(env) != 0;
    if (c->plan_groups == 0) c->use_groups = false;
    if (c->opt.precision == MRF_PREC_BF16 && !c->use_groups)
        return fail(c, MRF_ERANGE, "bf16 message storage needs the pipelined ray kernel (rays of at most %d edges)",
                    kThreads * 16 - 8);
    if (c->use_groups) {
        Scratch ka(c), kb(c), vt(c), ws(c);
        TRY(ensure(c, ka, (size_t)(E + 1) * 4, false));
        TRY(ensure(c, kb, (size_t)(E + 1) * 4, false));
        TRY(ensure(c, vt, (size_t)(E + 1) * 4, false));
        size_t wsb = sort_workspace_bytes(E);
        const size_t swb = scan_workspace_bytes(E);
        if (swb > wsb) wsb = swb;
        TRY(ensure(c, ws, wsb, false));
        TRY(build_groups(c, ptr<uint32_t>(ka), ptr<uint32_t>(kb), ptr<uint32_t>(vt), ws));
        release(c, ka);
        release(c, kb);
        release(c, vt);
        release(c, ws);
    }
    // rays for the FP64 accumulations (listed on the host)
    c->n_long = 0;
    if (c->opt.long_ray_f64 > 0 && c->max_len > c->opt.long_ray_f64) {
        std::vector<int64_t> ro((size_t)c->R + 1);
        CUDA_TRY(c, cudaMemcpyAsync(ro.data(), c->ray_off.p, ro.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        std::vector<uint32_t> ids;
        std::vector<int64_t> off(1, 0);
        for (int64_t r = 0; r < c->R; ++r)
            if (ro[r + 1] - ro[r] > c->opt.long_ray_f64) {
                ids.push_back((uint32_t)r);
                off.push_back(off.back() + (ro[r + 1] - ro[r]));
            }
        c->n_long = (int64_t)ids.size();
        TRY(ensure(c, c->lr_ids, ids.size() * 4, false));
        TRY(ensure(c, c->lr_off, off.size() * 8, false));
        TRY(ensure(c, c->lr_out, (size_t)off.back() * 4, false));
        TRY(ensure(c, c->lr_scr, (size_t)off.back() * 8, false));
        CUDA_TRY(c, cudaMemcpyAsync(c->lr_ids.p, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->lr_off.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the vectors go out of scope
    }
    // the per-edge transpose, where a path needs it
    if (!c->use_groups || c->opt.precision == MRF_PREC_F64 || c->opt.variants || c->opt.debug_checks)
        TRY(build_edge_transpose(c));
    if (c->opt.variants & MRF_VAR_KEYFRAME_AVG) TRY(build_pairs(c));
    // message storage
    if (c->opt.precision == MRF_PREC_F64) {
        TRY(ensure(c, c->lam64, (size_t)(E + kPad) * 8, false));
        TRY(ensure(c, c->bscr64, (size_t)(E + kPad) * 8, false));
    } else {
        TRY(ensure(c, c->lam, (size_t)(E + kPad) * (c->opt.precision == MRF_PREC_BF16 ? 2 : 4), false));
        // the log-domain ablation keeps log B per edge in the FP64 form's scratch
        if (c->opt.precision == MRF_PREC_F32_LOG) TRY(ensure(c, c->bscr64, (size_t)(E + kPad) * 8, false));
    }
    TRY(trim_pool(c));
    c->dirty = false;
    return MRF_OK;
}

// The transpose with the per-edge part, for the calls that read it.
int ensure_edge_transpose(mrf_ctx *c) {
    if (c->dirty) TRY(build_transpose(c));
    if (!c->have_perm && c->E > 0) {
        Prof prof(c, K_BUILD);
        TRY(build_edge_transpose(c));
        TRY(trim_pool(c));
    }
    return MRF_OK;
}

// Checks a frame's arguments and fills the traversal parameters and tables.
int trav_params(mrf_ctx *c, int scene, const float *depth_dev, int32_t W, int32_t H, const double pose[12],
                const mrf_intrinsics *K, const mrf_noise_lut *lut, TravParams &P, TravTables &TT) {
    if (scene < 0 || scene >= (int)c->scenes.size()) return fail(c, MRF_EINVAL, "scene %d out of range", scene);
    const mrf_grid &G = c->scenes[scene].g;
    const GridMap &GM = c->scenes[scene].gm;
    if (!depth_dev || !pose || !K || !lut) return fail(c, MRF_EINVAL, "null argument");
    if (W <= 0 || H <= 0) return fail(c, MRF_EINVAL, "frame size %dx%d", W, H);
    if (lut->n_bins < 2 || lut->n_bins > kMaxBins || !lut->log_sigma)
        return fail(c, MRF_EINVAL, "noise table needs 2..%d bins", kMaxBins);
    if (!(lut->d_hi > lut->d_lo) || !(lut->outlier_w >= 0.f && lut->outlier_w < 1.f))
        return fail(c, MRF_EINVAL, "noise table range or outlier weight out of range");
    if (!(K->fx != 0.f && K->fy != 0.f)) return fail(c, MRF_EINVAL, "zero focal length");
    for (int i = 0; i < 12; ++i)
        if (!isfinite(pose[i])) return fail(c, MRF_EINVAL, "non-finite pose");
    memset(&P, 0, sizeof P);
    P.nx = G.nx;
    P.nbx = GM.nbx;
    P.nby = GM.nby;
    P.key_base = (uint32_t)c->scenes[scene].key_base;
    P.ny = G.ny;
    P.nz = G.nz;
    P.h = G.res;
    for (int a = 0; a < 3; ++a) {
        P.o[a] = (float)((pose[a * 4 + 3] - (double)G.origin[a]) / (double)G.res);
        for (int b = 0; b < 3; ++b) P.R[a * 3 + b] = (float)pose[a * 4 + b];
    }
    P.fx = K->fx;
    P.fy = K->fy;
    P.cx = K->cx;
    P.cy = K->cy;
    P.W = W;
    P.H = H;
    P.n_bins = lut->n_bins;
    P.dlo = lut->d_lo;
    P.inv_delta = (float)((double)lut->n_bins / ((double)lut->d_hi - (double)lut->d_lo));
    P.w1 = 1.0f - lut->outlier_w;
    P.w_floor = (float)((double)lut->outlier_w / (double)lut->d_hi);
    P.dlo_d = lut->d_lo;
    P.delta_d = ((double)lut->d_hi - (double)lut->d_lo) / lut->n_bins;
    P.w_d = lut->outlier_w;
    P.floor_d = (double)lut->outlier_w / (double)lut->d_hi;
    P.has_bias = lut->bias != nullptr;
    for (int k = 0; k < lut->n_bins; ++k) {
        TT.log_sigma[k] = lut->log_sigma[k];
        TT.sig[k] = (float)exp((double)lut->log_sigma[k]);
        TT.bias[k] = lut->bias ? lut->bias[k] : 0.f;
    }
    // far-edge bounds: with sigma in [s_lo, s_hi] over the nodes k-1 .. k+2,
    // (1 - w) N <= (1 - w) exp(-x^2 / (2 s_hi^2)) / (s_lo sqrt(2 pi)); ask for
    // a term below floor * 2^-30 / e.  The shortcut is exact when floor and
    // floor (1 + 2^-30) round to the same float (no bias table: b would widen x).
    const double fl = P.floor_d;
    P.far_ok = P.w_d > 0.0 && !P.has_bias && fl > 0.0 && (float)fl == (float)(fl * (1.0 + 0x1p-30));
    for (int k = 0; k < lut->n_bins && P.far_ok; ++k) {
        double s_lo = HUGE_VAL, s_hi = 0.0;
        for (int j = k - 1; j <= k + 2; ++j) {
            const int jj = j < 0 ? 0 : (j > lut->n_bins - 1 ? lut->n_bins - 1 : j);
            const double s = exp((double)lut->log_sigma[jj]);
            s_lo = fmin(s_lo, s);
            s_hi = fmax(s_hi, s);
        }
        const double thr = -log(s_lo) - 0.91893853320467274178 + log1p(-P.w_d) - log(fl) + 30.0 * log(2.0) + 1.0;
        if (!(s_hi > 0.0 && s_hi < 1e30 && s_lo > 1e-30 && thr < 1e30)) {
            P.far_ok = 0;
            break;
        }
        TT.far_inv_sig[k] = (float)(1.0 / s_hi * (1.0 - 1e-6));
        TT.far_thr[k] = (float)(thr > 0.0 ? thr * (1.0 + 1e-6) : thr * (1.0 - 1e-6));
    }
    return MRF_OK;
}

int add_frame_impl(mrf_ctx *c, int scene, const float *depth_dev, int32_t W, int32_t H, const double pose[12],
                   const mrf_intrinsics *K, const mrf_noise_lut *lut) {
    Prof prof(c, K_TRAV);
    const int64_t npix = (int64_t)W * H;
    TravParams P;
    static thread_local TravTables TT;
    TRY(trav_params(c, scene, depth_dev, W, H, pose, K, lut, P, TT));
    if (c->nu_bg < 0.0) c->nu_bg = c->opt.nu_bg >= 0.f ? (double)c->opt.nu_bg : P.floor_d;
    // every nu of this frame is (1 - w) N + w / d_hi >= w / d_hi in FP64, and
    // rounding to float keeps the order
    c->nu_floor = fminf(c->nu_floor, (float)P.floor_d);
    {
        double smin = HUGE_VAL;
        for (int k = 0; k < lut->n_bins; ++k) smin = fmin(smin, exp((double)lut->log_sigma[k]));
        const double nmax = (1.0 - P.w_d) / (2.5066282746310002 * smin) + P.floor_d;
        if (!(nmax <= c->nu_max)) c->nu_max = nmax;   // also takes a NaN or inf bound
    }
    // ray set-up: per-pixel edge counts and ranges
    const bool f64 = c->opt.precision == MRF_PREC_F64;
    if (c->R + npix + 1 > c->cap_R) {
        int64_t nc = c->cap_R + c->cap_R / 2;
        if (nc < c->R + npix + 1) nc = c->R + npix + 1;
        TRY(ensure(c, c->ray_off, (size_t)(nc + 1) * 8, true));
        TRY(ensure(c, c->Zr, (size_t)nc * 4, true));
        c->cap_R = nc;
    }
    TRY(ensure(c, c->counts, (size_t)npix * 4, false));
    TRY(ensure(c, c->rsetup, (size_t)npix * kRaySetupBytes, false));
    TRY(ensure(c, c->scan_ws, scan_workspace_bytes(npix), false));
    CUDA_TRY(c, cudaMemsetAsync(c->maxlen_dev.p, 0, 4, c->stream));
    CUDA_TRY(c, launch_ray_setup(P, TT, depth_dev, ptr<int32_t>(c->counts), ptr<float>(c->Zr) + c->R,
                                 ptr<int32_t>(c->maxlen_dev), c->rsetup.p, c->stream));
    CUDA_TRY(c, exclusive_scan_i32_i64(ptr<int32_t>(c->counts), ptr<int64_t>(c->ray_off) + c->R, npix, c->E,
                                       c->scan_ws.p, c->stream));
    c->launches += 4;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<int64_t>(c->ray_off) + c->R + npix, 8, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned + 1, c->maxlen_dev.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t newE = c->h_pinned[0];
    const int32_t ml = (int32_t)(c->h_pinned[1] & 0xffffffff);
    if (newE >= ((int64_t)1 << 32) - kPad)
        return fail(c, MRF_ERANGE, "%lld edges exceed the 2^32 edge limit", (long long)newE);
    if (newE + kPad > c->cap_E) {
        int64_t nc = c->cap_E + c->cap_E / 2;
        if (nc < newE + kPad) nc = newE + kPad;
        TRY(ensure(c, c->vox, (size_t)nc * 4, true));
        TRY(ensure(c, c->dmid, (size_t)nc * 4, true));
        if (f64) TRY(ensure(c, c->nu64, (size_t)nc * 8, true));
        else TRY(ensure(c, c->nu, (size_t)nc * 4, true));
        if (c->opt.variants & MRF_VAR_LENGTH_WEIGHT) TRY(ensure(c, c->wlen, (size_t)nc * 4, true));
        // the slack after the edges is read (and ignored) by full-width tile
        // loads and gathers: keep its likelihoods finite and its voxel keys
        // valid (the ray kernel gathers T at every window position)
        if (!f64) CUDA_TRY(c, cudaMemsetAsync(ptr<float>(c->nu) + newE, 0, (size_t)(nc - newE) * 4, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(ptr<uint32_t>(c->vox) + newE, 0, (size_t)(nc - newE) * 4, c->stream));
        c->cap_E = nc;
    }
    CUDA_TRY(c, launch_ray_walk(P, TT, c->rsetup.p, ptr<int64_t>(c->ray_off) + c->R, ptr<uint32_t>(c->vox),
                                ptr<float>(c->dmid), f64 ? nullptr : ptr<float>(c->nu),
                                f64 ? ptr<double>(c->nu64) : nullptr,
                                (c->opt.variants & MRF_VAR_LENGTH_WEIGHT) ? ptr<float>(c->wlen) : nullptr, c->stream));
    c->launches += 1;
    c->frame_E.push_back(c->E);
    c->R += npix;
    c->E = newE;
    if (ml > c->max_len) c->max_len = ml;
    c->n_frames += 1;
    c->dirty = true;
    return MRF_OK;
}

// ck_lam / ck_T (optional, FP32 contexts): after pass t (1-based) the messages
// go to ck_lam + (t-1) E and the voxel totals to ck_T + (t-1) Vk.
int infer_impl(mrf_ctx *c, int32_t iters, float *ck_lam = nullptr, float *ck_T = nullptr) {
    if (iters < 0) return fail(c, MRF_EINVAL, "iters = %d", iters);
    if (c->dirty) TRY(build_transpose(c));
    const double gamma = c->prior;
    const double lp = log(gamma) - log1p(-gamma);
    const double ip = c->opt.init_p > 0.f ? (double)c->opt.init_p : gamma;
    const double L0 = log(ip) - log1p(-ip);
    const bool f64 = c->opt.precision == MRF_PREC_F64;
    {
        Prof prof(c, K_OTHER);
        if (f64) {
            TRY(ensure(c, c->T64, (size_t)c->Vk * 8, false));
            CUDA_TRY(c, launch_fill_f64(ptr<double>(c->T64), c->Vk, lp, c->stream));
        } else {
            TRY(ensure(c, c->T, (size_t)c->Vk * 4, false));
            CUDA_TRY(c, launch_fill_f32(ptr<float>(c->T), c->Vk, (float)lp, c->stream));
        }
        c->launches += 1;
    }
    if (c->E == 0) return MRF_OK;
    // the FP32 kernels carry likelihoods as excesses over a floor no nu and
    // not nu_bg is below
    const float nu_ref = fminf((float)c->nu_bg, c->nu_floor);
    // messages need no range, NaN or clamp handling when the floor is positive
    // and the likelihoods are bounded well inside FP32 (message() in ray_tile.cuh)
    const bool floored = nu_ref >= 1e-30f && c->nu_max < 1e29 && c->nu_max < 1e25 * (double)nu_ref &&
                         c->nu_bg < 1e29 && c->nu_bg < 1e25 * (double)nu_ref;
    for (int it = 0; it < iters; ++it) {
        const int first = it == 0;
        if (f64) {
            {
                Prof prof(c, K_RAY);
                CUDA_TRY(c, launch_ray_messages_f64(ptr<int64_t>(c->ray_off), c->R, ptr<uint32_t>(c->vox),
                                                    ptr<double>(c->nu64), ptr<double>(c->T64), ptr<double>(c->lam64),
                                                    ptr<double>(c->bscr64), c->nu_bg, first, L0, c->stream));
            }
            {
                Prof prof(c, K_RED);
                CUDA_TRY(c, launch_voxel_reduce_f64(ptr<uint32_t>(c->perm), ptr<uint32_t>(c->seg_off),
                                                    ptr<uint32_t>(c->seg_vox), ptr<uint32_t>(c->red_plan),
                                                    c->n_red_tiles, ptr<double>(c->lam64), ptr<double>(c->T64), lp,
                                                    c->E, ptr<double>(c->head_part),
                                                    ptr<double>(c->tail_part), ptr<uint32_t>(c->tail_seg), c->stream));
            }
        } else {
            {
                Prof prof(c, K_RAY);
                if (c->n_long)   // before the FP32 kernel overwrites the old messages it reads
                    CUDA_TRY(c, launch_long_rays_f64(ptr<int64_t>(c->ray_off), ptr<uint32_t>(c->lr_ids), c->n_long,
                                                     ptr<int64_t>(c->lr_off), ptr<uint32_t>(c->vox),
                                                     ptr<float>(c->nu), ptr<float>(c->T), ptr<float>(c->lam), first,
                                                     (double)(float)L0, c->nu_bg, ptr<float>(c->lr_out),
                                                     ptr<double>(c->lr_scr),
                                                     c->stream));
                if (c->use_pipe) {
                    CUDA_TRY(c, launch_ray_pipe(c->kt, c->pipe_nt, c->opt.precision == MRF_PREC_BF16,
                                                (int64_t)c->n_sm, ptr<int64_t>(c->tile_E),
                                                c->n_ray_tiles, ptr<uint32_t>(c->ray_starts), ptr<uint32_t>(c->vox),
                                                ptr<float>(c->nu), ptr<float>(c->T), c->lam.p,
                                                (float)c->nu_bg, nu_ref, first, (float)L0, ptr<uint32_t>(c->err_dev),
                                                c->use_groups ? ptr<uint16_t>(c->g_lidx) : nullptr,
                                                c->use_groups ? ptr<uint32_t>(c->g_ends) : nullptr,
                                                c->use_groups ? ptr<uint16_t>(c->g_gid) : nullptr,
                                                c->use_groups ? ptr<uint32_t>(c->g_key) : nullptr,
                                                c->use_groups ? ptr<int64_t>(c->g_tg_off) : nullptr,
                                                c->use_groups ? ptr<float>(c->g_partial) : nullptr, c->stream,
                                                floored));
                } else if (c->opt.precision == MRF_PREC_F32_LOG) {
                    CUDA_TRY(c, launch_ray_messages_log32(ptr<int64_t>(c->ray_off), c->R, ptr<uint32_t>(c->vox),
                                                          ptr<float>(c->nu), ptr<float>(c->T), ptr<float>(c->lam),
                                                          ptr<float>(c->bscr64), (float)c->nu_bg, first, (float)L0,
                                                          c->stream));
                } else {
                    CUDA_TRY(c, launch_ray_messages_f32(c->kt, ptr<int64_t>(c->ray_off), ptr<uint32_t>(c->ray_plan),
                                                        c->n_ray_tiles, ptr<uint32_t>(c->vox), ptr<float>(c->nu),
                                                        ptr<float>(c->T), ptr<float>(c->lam), c->E + kPad,
                                                        (float)c->nu_bg, nu_ref, first, (float)L0, nullptr,
                                                        c->stream,
                                                        (c->opt.variants & MRF_VAR_LENGTH_WEIGHT)
                                                            ? ptr<float>(c->wlen) : nullptr));
                }
            }
            if (c->n_long) {
                Prof prof(c, K_RAY);
                CUDA_TRY(c, launch_long_scatter(ptr<int64_t>(c->ray_off), ptr<uint32_t>(c->lr_ids), c->n_long,
                                                ptr<int64_t>(c->lr_off), ptr<float>(c->lr_out), ptr<float>(c->lam),
                                                c->stream));
                c->launches += 2;
            }
            if (c->use_groups) {
                Prof prof(c, K_RED);
                CUDA_TRY(c, launch_voxel_reduce_f32(ptr<uint32_t>(c->g_tp2), ptr<uint32_t>(c->g_seg_off2),
                                                    ptr<uint32_t>(c->seg_vox), ptr<uint32_t>(c->g_plan), c->n_red2,
                                                    ptr<float>(c->g_partial), ptr<float>(c->T), (float)lp,
                                                    c->n_groups, ptr<float>(c->g_head), ptr<float>(c->g_tail),
                                                    ptr<uint32_t>(c->g_tseg), c->stream));
            } else {
                Prof prof(c, K_RED);
                CUDA_TRY(c, launch_voxel_reduce_f32(ptr<uint32_t>(c->perm), ptr<uint32_t>(c->seg_off),
                                                    ptr<uint32_t>(c->seg_vox), ptr<uint32_t>(c->red_plan),
                                                    c->n_red_tiles, ptr<float>(c->lam), ptr<float>(c->T), (float)lp,
                                                    c->E, ptr<float>(c->head_part),
                                                    ptr<float>(c->tail_part), ptr<uint32_t>(c->tail_seg), c->stream));
            }
        }
        c->launches += 3;
        if (c->opt.variants & MRF_VAR_KEYFRAME_AVG) {
            Prof prof(c, K_OTHER);
            CUDA_TRY(c, launch_voxel_reduce_f32(ptr<uint32_t>(c->perm), ptr<uint32_t>(c->pair_off),
                                                ptr<uint32_t>(c->pair_ident), ptr<uint32_t>(c->pair_plan),
                                                c->n_pair_tiles, ptr<float>(c->lam), ptr<float>(c->pair_sum), 0.f,
                                                c->E, ptr<float>(c->pair_head), ptr<float>(c->pair_tail),
                                                ptr<uint32_t>(c->pair_tseg), c->stream));
            CUDA_TRY(c, launch_pair_scatter(ptr<uint32_t>(c->perm), ptr<uint32_t>(c->pair_pid),
                                            ptr<uint32_t>(c->pair_off), ptr<float>(c->pair_sum), c->E,
                                            ptr<float>(c->lam), c->stream));
            c->launches += 3;
        }
        if (ck_lam && !f64) {
            CUDA_TRY(c, cudaMemcpyAsync(ck_lam + (size_t)it * c->E, c->lam.p, (size_t)c->E * 4,
                                        cudaMemcpyDeviceToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(ck_T + (size_t)it * c->Vk, c->T.p, (size_t)c->Vk * 4,
                                        cudaMemcpyDeviceToDevice, c->stream));
        }
    }
    return MRF_OK;
}

// Voxel-major view of n edge keys (stable sort, segments, reduction plan) into
// the given buffers; *S receives the number of segments, *ntiles the plan's.
int edge_transpose(mrf_ctx *c, const uint32_t *keys, int64_t n, Buf &perm, Buf &seg_off, Buf &seg_vox, Buf &plan,
                   int64_t *S_out, int64_t *ntiles_out) {
    Scratch ka(c), kb(c), vt(c), ws(c);
    TRY(ensure(c, perm, (size_t)(n + kPad) * 4, false));
    TRY(ensure(c, ka, (size_t)(n + 1) * 4, false));
    TRY(ensure(c, kb, (size_t)(n + 1) * 4, false));
    TRY(ensure(c, vt, (size_t)(n + 1) * 4, false));
    size_t wsb = sort_workspace_bytes(n);
    const size_t swb = scan_workspace_bytes(n);
    if (swb > wsb) wsb = swb;
    TRY(ensure(c, ws, wsb, false));
    uint32_t *sorted = nullptr;
    CUDA_TRY(c, radix_sort_edges(keys, key_bits(c->Vk), n, ptr<uint32_t>(ka), ptr<uint32_t>(kb), ptr<uint32_t>(vt),
                                 ptr<uint32_t>(perm), &sorted, ws.p, c->stream, &c->launches));
    uint32_t *flags = sorted == ptr<uint32_t>(ka) ? ptr<uint32_t>(kb) : ptr<uint32_t>(ka);
    CUDA_TRY(c, segment_heads(sorted, n, flags, c->stream));
    CUDA_TRY(c, exclusive_scan_u32(flags, ptr<uint32_t>(vt), n, ws.p, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<uint32_t>(vt) + n, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t S = (int64_t)(*(uint32_t *)c->h_pinned);
    TRY(ensure(c, seg_off, (size_t)(S + 1) * 4, false));
    TRY(ensure(c, seg_vox, (size_t)(S > 0 ? S : 1) * 4, false));
    CUDA_TRY(c, segment_emit(sorted, ptr<uint32_t>(vt), n, ptr<uint32_t>(seg_off), ptr<uint32_t>(seg_vox), c->stream));
    const int64_t nt = ceil_div(n, kTile);
    TRY(ensure(c, plan, (size_t)(nt > 0 ? nt : 1) * 8, false));
    CUDA_TRY(c, launch_reduce_plan(ptr<uint32_t>(seg_off), S, n, ptr<uint32_t>(plan), nt, c->stream));
    c->launches += 4;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    release(c, ka);
    release(c, kb);
    release(c, vt);
    release(c, ws);
    *S_out = S;
    *ntiles_out = nt;
    return MRF_OK;
}

// Reads (and clears) the device error word after a synchronisation point.
int device_errors(mrf_ctx *c) {
    uint32_t e = 0;
    CUDA_TRY(c, cudaMemcpy(&e, c->err_dev.p, 4, cudaMemcpyDeviceToHost));
    if (e == 0) return MRF_OK;
    CUDA_TRY(c, cudaMemset(c->err_dev.p, 0, 4));
    return fail(c, MRF_ETIMEOUT, "a bounded device-side wait gave up (code %u)", e);
}

void free_all(mrf_ctx *c) {
    Buf *bufs[] = {&c->ray_off, &c->Zr, &c->vox, &c->dmid, &c->nu, &c->nu64, &c->perm, &c->seg_off, &c->seg_vox,
                   &c->lam, &c->T, &c->lam64, &c->T64, &c->bscr64, &c->ray_plan, &c->red_plan, &c->head_part,
                   &c->tail_part, &c->tail_seg, &c->counts, &c->rsetup, &c->maxlen_dev, &c->scan_ws, &c->depth_stage,
                   &c->tile_E, &c->ray_starts, &c->err_dev, &c->g_lidx, &c->g_ends, &c->g_gid, &c->g_key, &c->g_tg_off, &c->g_tp2,
                   &c->g_seg_off2, &c->g_partial, &c->g_plan, &c->g_head, &c->g_tail, &c->g_tseg,
                   &c->h_ray_off, &c->h_Zr, &c->h_vox, &c->h_dmid, &c->gr_ck_lam, &c->gr_ck_T, &c->gr_gT,
                   &c->gr_glam, &c->gr_gL, &c->gr_gLn, &c->gr_gnu, &c->gr_sP, &c->gr_sA, &c->gr_sB, &c->gr_sg,
                   &c->gr_gbg, &c->gr_head, &c->gr_tail, &c->gr_tseg, &c->gr_part, &c->gr_hQ, &c->gr_hnu,
                   &c->gr_hgp, &c->gr_hgnu, &c->gr_hloss, &c->gr_hgbg, &c->gr_hperm, &c->gr_hso, &c->gr_hsv,
                   &c->gr_hplan, &c->ac_ray_off, &c->ac_Z, &c->ac_vox, &c->ac_tin, &c->ac_tout, &c->ac_cnt,
                   &c->wlen, &c->pair_off, &c->frame_E_dev, &c->pair_pid, &c->pair_ident, &c->pair_sum,
                   &c->pair_plan, &c->pair_head, &c->pair_tail, &c->pair_tseg, &c->lr_ids, &c->lr_off,
                   &c->lr_out, &c->lr_scr};
    for (Buf *b : bufs) release(c, *b);
}

int create_impl(mrf_ctx **out, int32_t n, const mrf_grid *grids, float prior, const mrf_options *opt,
                void *cuda_stream) {
    if (!out || !grids || n <= 0) return MRF_EINVAL;
    *out = nullptr;
    std::vector<mrf_ctx::Scene> sc((size_t)n);
    int64_t V = 0, Vk = 0;
    for (int32_t i = 0; i < n; ++i) {
        const mrf_grid *g = grids + i;
        if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || !(g->res > 0.f)) return MRF_EINVAL;
        const int64_t nb[3] = {(g->nx + 7) / 8, (g->ny + 7) / 8, (g->nz + 7) / 8};
        sc[i].g = *g;
        sc[i].gm = {(uint32_t)g->nx, (uint32_t)g->ny, (uint32_t)g->nz, (uint32_t)nb[0], (uint32_t)nb[1]};
        sc[i].V = (int64_t)g->nx * g->ny * g->nz;
        sc[i].key_base = Vk;
        sc[i].lin_base = V;
        V += sc[i].V;
        Vk += nb[0] * nb[1] * nb[2] * 512;
        if (V >= ((int64_t)1 << 32) || Vk >= ((int64_t)1 << 32)) return MRF_ERANGE;
    }
    const mrf_grid *g = grids;
    if (!(prior > 0.f && prior < 1.f)) return MRF_EINVAL;
    mrf_options o;
    mrf_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != MRF_PREC_F32 && o.precision != MRF_PREC_F64 && o.precision != MRF_PREC_BF16 &&
        o.precision != MRF_PREC_F32_LOG)
        return MRF_EINVAL;
    if ((o.variants & ~(MRF_VAR_LENGTH_WEIGHT | MRF_VAR_KEYFRAME_AVG)) ||
        (o.variants && o.precision != MRF_PREC_F32))
        return MRF_EINVAL;
    if (o.long_ray_f64 < 0 || (o.long_ray_f64 > 0 && (o.precision != MRF_PREC_F32 || o.variants)))
        return MRF_EINVAL;
    if (!(o.init_p < 1.f)) return MRF_EINVAL;
    mrf_ctx *c = new (std::nothrow) mrf_ctx();
    if (!c) return MRF_ENOMEM;
    c->g = *g;
    c->prior = prior;
    c->opt = o;
    c->V = V;
    c->Vk = Vk;
    c->scenes = sc;
    c->gm = sc[0].gm;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return MRF_ECUDA;
    }
    {   // keep freed pool memory for reuse by the next build instead of returning it at every sync
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (cudaMallocHost((void **)&c->h_pinned, 4 * sizeof(int64_t)) != cudaSuccess) {
        delete c;
        return MRF_ENOMEM;
    }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (c->n_sm <= 0) c->n_sm = 1;
    if (ensure(c, c->err_dev, 16, false) != MRF_OK || cudaMemsetAsync(c->err_dev.p, 0, 16, c->stream) != cudaSuccess) {
        cudaFreeHost(c->h_pinned);
        delete c;
        return MRF_ENOMEM;
    }
    if (ensure(c, c->maxlen_dev, 16, false) != MRF_OK) {
        cudaFreeHost(c->h_pinned);
        delete c;
        return MRF_ENOMEM;
    }
    *out = c;
    return MRF_OK;
}

}  // namespace

extern "C" {

void mrf_default_options(mrf_options *opt) {
    if (!opt) return;
    opt->precision = MRF_PREC_F32;
    opt->nu_bg = -1.f;
    opt->init_p = 0.f;
    opt->debug_checks = 0;
    opt->variants = 0;
    opt->long_ray_f64 = 0;
}

int mrf_create(mrf_ctx **out, const mrf_grid *g, float prior, const mrf_options *opt, void *cuda_stream) {
    return create_impl(out, 1, g, prior, opt, cuda_stream);
}

int mrf_create_batch(mrf_ctx **out, int32_t n_scenes, const mrf_grid *grids, float prior, const mrf_options *opt,
                     void *cuda_stream) {
    return create_impl(out, n_scenes, grids, prior, opt, cuda_stream);
}

int mrf_scene_count(mrf_ctx *c, int32_t *n_scenes, int64_t *n_voxels) {
    if (!c) return MRF_EINVAL;
    if (n_scenes) *n_scenes = (int32_t)c->scenes.size();
    if (n_voxels) *n_voxels = c->V;
    return MRF_OK;
}

void mrf_destroy(mrf_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    cudaStreamSynchronize(c->stream);
    {   // the context's memory goes back to the device
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    }
    for (auto &ev : c->events) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (auto e : c->gev)
        if (e) cudaEventDestroy(e);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
}

int mrf_reset(mrf_ctx *c) {
    TRY(check_ctx(c));
    c->R = 0;
    c->E = 0;
    c->max_len = 0;
    c->n_frames = 0;
    c->n_seg = 0;
    c->nu_bg = -1.0;
    c->nu_floor = FLT_MAX;
    c->nu_max = 0.0;
    c->hR = 0;
    c->hE = 0;
    c->frame_E.clear();
    c->n_pairs = 0;
    c->dirty = true;
    return MRF_OK;
}

int mrf_set_stream(mrf_ctx *c, void *s) {
    TRY(check_ctx(c));
    c->stream = (cudaStream_t)s;
    return MRF_OK;
}

int mrf_add_frame(mrf_ctx *c, const float *depth_dev, int32_t W, int32_t H, const double cam_to_world[12],
                  const mrf_intrinsics *K, const mrf_noise_lut *lut) {
    TRY(check_ctx(c));
    return add_frame_impl(c, 0, depth_dev, W, H, cam_to_world, K, lut);
}

int mrf_add_frame_to(mrf_ctx *c, int32_t scene, const float *depth_dev, int32_t W, int32_t H,
                     const double cam_to_world[12], const mrf_intrinsics *K, const mrf_noise_lut *lut) {
    TRY(check_ctx(c));
    return add_frame_impl(c, scene, depth_dev, W, H, cam_to_world, K, lut);
}

int mrf_add_frame_host(mrf_ctx *c, const float *depth_host, int32_t W, int32_t H, const double cam_to_world[12],
                       const mrf_intrinsics *K, const mrf_noise_lut *lut) {
    TRY(check_ctx(c));
    if (!depth_host || W <= 0 || H <= 0) return fail(c, MRF_EINVAL, "bad host depth frame");
    const size_t bytes = (size_t)W * H * 4;
    TRY(ensure(c, c->depth_stage, bytes, false));
    CUDA_TRY(c, cudaMemcpyAsync(c->depth_stage.p, depth_host, bytes, cudaMemcpyHostToDevice, c->stream));
    return add_frame_impl(c, 0, ptr<float>(c->depth_stage), W, H, cam_to_world, K, lut);
}

int mrf_infer(mrf_ctx *c, int32_t iters) {
    TRY(check_ctx(c));
    return infer_impl(c, iters);
}

int mrf_marginals(mrf_ctx *c, float *out_dev) {
    TRY(check_ctx(c));
    if (!out_dev) return fail(c, MRF_EINVAL, "null output");
    Prof prof(c, K_OTHER);
    const bool f64 = c->opt.precision == MRF_PREC_F64;
    if (f64 ? !c->T64.p : !c->T.p) return fail(c, MRF_ESTATE, "marginals before infer");
    for (const auto &sc : c->scenes) {   // scenes in order, each x fastest
        if (f64)
            CUDA_TRY(c, launch_marginals_f64(ptr<double>(c->T64) + sc.key_base, out_dev + sc.lin_base, sc.gm,
                                             c->stream));
        else
            CUDA_TRY(c, launch_marginals_f32(ptr<float>(c->T) + sc.key_base, out_dev + sc.lin_base, sc.gm,
                                             c->stream));
        c->launches += 1;
    }
    return MRF_OK;
}

int mrf_marginals_host(mrf_ctx *c, float *out_host) {
    TRY(check_ctx(c));
    if (!out_host) return fail(c, MRF_EINVAL, "null output");
    Scratch tmp(c);
    TRY(ensure(c, tmp, (size_t)c->V * 4, false));
    int r = mrf_marginals(c, ptr<float>(tmp));
    if (r == MRF_OK) {
        cudaError_t e = cudaMemcpyAsync(out_host, tmp.p, (size_t)c->V * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) r = fail(c, MRF_ECUDA, "marginals copy: %s", cudaGetErrorString(e));
        else r = device_errors(c);
    }
    release(c, tmp);
    return r;
}

int mrf_stats(mrf_ctx *c, int64_t *n_rays, int64_t *n_edges) {
    if (!c) return MRF_EINVAL;
    if (n_rays) *n_rays = c->R;
    if (n_edges) *n_edges = c->E;
    return MRF_OK;
}

int mrf_stats2(mrf_ctx *c, int32_t *max_ray_len, int64_t *n_touched) {
    if (!c) return MRF_EINVAL;
    if (max_ray_len) *max_ray_len = c->max_len;
    if (n_touched) *n_touched = c->dirty ? -1 : c->n_seg;
    return MRF_OK;
}

int mrf_plan_info(mrf_ctx *c, int32_t *ray_items, int64_t *n_ray_tiles, int64_t *n_groups) {
    if (!c) return MRF_EINVAL;
    if (ray_items) *ray_items = c->dirty ? -1 : c->kt;
    if (n_ray_tiles) *n_ray_tiles = c->dirty ? -1 : c->n_ray_tiles;
    if (n_groups) *n_groups = c->dirty ? -1 : (c->use_groups ? c->n_groups : 0);
    return MRF_OK;
}

int mrf_synchronize(mrf_ctx *c) {
    TRY(check_ctx(c));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return device_errors(c);
}

int mrf_debug_fail_alloc(mrf_ctx *c, int64_t nth) {
    TRY(check_ctx(c));
    if (nth < 0) return fail(c, MRF_EINVAL, "nth = %lld", (long long)nth);
    c->fail_alloc_at = nth;
    c->alloc_count = 0;
    return MRF_OK;
}

int mrf_debug_wait_probe(mrf_ctx *c) {
    TRY(check_ctx(c));
    CUDA_TRY(c, launch_wait_probe(ptr<uint32_t>(c->err_dev), c->stream));
    c->launches += 1;
    return MRF_OK;
}

const char *mrf_last_error(mrf_ctx *c) {
    static thread_local std::string last;
    if (!c) return "null context";
    last = c->err;
    c->err.clear();
    c->sticky = MRF_OK;
    return last.c_str();
}

int mrf_export_rays(mrf_ctx *c, int64_t *ray_off_dev, uint32_t *vox_dev, float *d_dev, float *Z_dev) {
    TRY(check_ctx(c));
    if (c->scenes.size() > 1) return fail(c, MRF_ESTATE, "voxel-indexed exports need a single-scene context");
    if (ray_off_dev) {
        if (c->R == 0) {
            CUDA_TRY(c, cudaMemsetAsync(ray_off_dev, 0, 8, c->stream));
        } else {
            CUDA_TRY(c, cudaMemcpyAsync(ray_off_dev, c->ray_off.p, (size_t)(c->R + 1) * 8, cudaMemcpyDeviceToDevice,
                                        c->stream));
        }
    }
    if (vox_dev && c->E) CUDA_TRY(c, launch_keys_to_linear(ptr<uint32_t>(c->vox), vox_dev, c->E, c->gm, c->stream));
    if (d_dev && c->E)
        CUDA_TRY(c, cudaMemcpyAsync(d_dev, c->dmid.p, (size_t)c->E * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (Z_dev && c->R)
        CUDA_TRY(c, cudaMemcpyAsync(Z_dev, c->Zr.p, (size_t)c->R * 4, cudaMemcpyDeviceToDevice, c->stream));
    return MRF_OK;
}

int mrf_export_nu(mrf_ctx *c, float *nu_dev) {
    TRY(check_ctx(c));
    if (!nu_dev || !c->E) return MRF_OK;
    if (c->opt.precision == MRF_PREC_F64) {
        CUDA_TRY(c, launch_f64_to_f32(ptr<double>(c->nu64), nu_dev, c->E, c->stream));
    } else {
        CUDA_TRY(c, cudaMemcpyAsync(nu_dev, c->nu.p, (size_t)c->E * 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    return MRF_OK;
}

int mrf_export_messages(mrf_ctx *c, float *lam_dev, float *T_dev) {
    TRY(check_ctx(c));
    if (c->scenes.size() > 1) return fail(c, MRF_ESTATE, "voxel-indexed exports need a single-scene context");
    if (c->opt.precision == MRF_PREC_F64) return fail(c, MRF_ESTATE, "context is FP64");
    if (lam_dev && c->E && c->lam.p) {
        if (c->opt.precision == MRF_PREC_BF16)
            CUDA_TRY(c, launch_bf16_to_f32(c->lam.p, lam_dev, c->E, c->stream));
        else
            CUDA_TRY(c, cudaMemcpyAsync(lam_dev, c->lam.p, (size_t)c->E * 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (T_dev && c->T.p) CUDA_TRY(c, launch_gather_linear_f32(ptr<float>(c->T), T_dev, c->gm, c->stream));
    return MRF_OK;
}

int mrf_export_messages_f64(mrf_ctx *c, double *lam_dev, double *T_dev) {
    TRY(check_ctx(c));
    if (c->scenes.size() > 1) return fail(c, MRF_ESTATE, "voxel-indexed exports need a single-scene context");
    if (c->opt.precision != MRF_PREC_F64) return fail(c, MRF_ESTATE, "context is not FP64");
    if (lam_dev && c->E && c->lam64.p)
        CUDA_TRY(c, cudaMemcpyAsync(lam_dev, c->lam64.p, (size_t)c->E * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (T_dev && c->T64.p) CUDA_TRY(c, launch_gather_linear_f64(ptr<double>(c->T64), T_dev, c->gm, c->stream));
    return MRF_OK;
}

int mrf_export_transpose(mrf_ctx *c, uint32_t *perm_dev, uint32_t *seg_off_dev, uint32_t *seg_vox_dev,
                         int64_t *n_seg) {
    TRY(check_ctx(c));
    if (c->scenes.size() > 1) return fail(c, MRF_ESTATE, "voxel-indexed exports need a single-scene context");
    TRY(ensure_edge_transpose(c));
    if (n_seg) *n_seg = c->n_seg;
    if (perm_dev && c->E)
        CUDA_TRY(c, cudaMemcpyAsync(perm_dev, c->perm.p, (size_t)c->E * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (seg_off_dev && c->E)
        CUDA_TRY(c, cudaMemcpyAsync(seg_off_dev, c->seg_off.p, (size_t)(c->n_seg + 1) * 4, cudaMemcpyDeviceToDevice,
                                    c->stream));
    if (seg_vox_dev && c->n_seg)
        CUDA_TRY(c, launch_keys_to_linear(ptr<uint32_t>(c->seg_vox), seg_vox_dev, c->n_seg, c->gm, c->stream));
    return MRF_OK;
}

int mrf_export_groups(mrf_ctx *c, int64_t *tile_E_dev, int64_t *tg_off_dev, uint16_t *lidx_dev, uint16_t *gid_dev,
                      uint32_t *ends_dev, uint32_t *gkey_dev, int64_t *n_tiles, int64_t *n_groups) {
    TRY(check_ctx(c));
    if (c->dirty) TRY(build_transpose(c));
    if (!c->use_groups && c->E > 0) return fail(c, MRF_ESTATE, "the context's plan has no group tables");
    const int64_t E = c->E, nt = c->n_ray_tiles, G = c->n_groups;
    if (n_tiles) *n_tiles = nt;
    if (n_groups) *n_groups = G;
    if (E == 0) return MRF_OK;
    auto copy = [&](void *dst, const Buf &src, size_t bytes) -> int {
        if (dst && bytes) CUDA_TRY(c, cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return MRF_OK;
    };
    TRY(copy(tile_E_dev, c->tile_E, (size_t)(nt + 1) * 8));
    TRY(copy(tg_off_dev, c->g_tg_off, (size_t)(nt + 1) * 8));
    TRY(copy(lidx_dev, c->g_lidx, (size_t)E * 2));
    TRY(copy(gid_dev, c->g_gid, (size_t)E * 2));
    TRY(copy(ends_dev, c->g_ends, (size_t)ceil_div(E, 32) * 4));
    TRY(copy(gkey_dev, c->g_key, (size_t)G * 4));
    return MRF_OK;
}

int mrf_profile_enable(mrf_ctx *c, int32_t on) {
    TRY(check_ctx(c));
    c->profiling = on != 0;
    return MRF_OK;
}

int mrf_profile_read(mrf_ctx *c, mrf_profile_times *out) {
    TRY(check_ctx(c));
    if (!out) return fail(c, MRF_EINVAL, "null output");
    memset(out, 0, sizeof *out);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (auto &ev : c->events) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.a, ev.b);
        switch (ev.kind) {
            case K_RAY: out->ms_ray_messages += ms; out->n_ray_messages++; break;
            case K_RED: out->ms_voxel_reduce += ms; out->n_voxel_reduce++; break;
            case K_OTHER: out->ms_other_infer += ms; out->n_other_infer++; break;
            case K_BUILD: out->ms_build += ms; out->n_build++; break;
            default: out->ms_traverse += ms; out->n_traverse++; break;
        }
        c->event_pool.push_back(ev.a);
        c->event_pool.push_back(ev.b);
    }
    c->events.clear();
    return device_errors(c);
}

int64_t mrf_launch_count(const mrf_ctx *c) { return c ? c->launches : 0; }

size_t mrf_ray_messages_workspace(int64_t n_rays, int64_t n_edges, int32_t max_ray_len) {
    (void)n_rays;
    const int kt = ray_tile_items(max_ray_len < 1 ? 1 : max_ray_len);
    if (kt == 0) return 0;
    const int64_t window = ray_tile_window(kt, max_ray_len < 1 ? 1 : max_ray_len);
    return (size_t)(ceil_div(n_edges > 0 ? n_edges : 1, window) + 2) * 4;
}

int mrf_ray_messages(const int64_t *ray_off_dev, int64_t n_rays, int32_t max_ray_len, const uint32_t *vox_dev,
                     const float *nu_dev, const float *T_dev, float *lam_dev, float nu_bg, int32_t first, float L0,
                     void *workspace_dev, size_t workspace_bytes, void *stream) {
    if (n_rays < 0 || !ray_off_dev || max_ray_len < 0) return MRF_EINVAL;
    if (n_rays >= ((int64_t)1 << 32) - 1) return MRF_ERANGE;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t E = 0;
    if (cudaMemcpyAsync(&E, ray_off_dev + n_rays, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MRF_ECUDA;
    if (E == 0) return MRF_OK;
    if (!vox_dev || !nu_dev || !lam_dev || (!first && !T_dev) || !workspace_dev) return MRF_EINVAL;
    const int kt = ray_tile_items(max_ray_len < 1 ? 1 : max_ray_len);
    if (kt == 0) return MRF_ERANGE;
    if (workspace_bytes < mrf_ray_messages_workspace(n_rays, E, max_ray_len)) return MRF_EINVAL;
    const int64_t window = ray_tile_window(kt, max_ray_len);
    const int64_t ntiles = ceil_div(E, window);
    uint32_t *plan = (uint32_t *)workspace_dev;
    uint32_t *err = plan + ntiles + 1;
    uint32_t h_err = 0;
    if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) return MRF_ECUDA;
    if (launch_ray_plan(ray_off_dev, n_rays, E, window, plan, ntiles, s) != cudaSuccess) return MRF_ECUDA;
    // the caller's likelihoods have no known floor: excesses over 0 (or over a
    // negative nu_bg, which the argument checks would have to allow)
    const float nu_ref = nu_bg < 0.f ? nu_bg : 0.f;
    if (launch_ray_messages_f32(kt, ray_off_dev, plan, ntiles, vox_dev, nu_dev, T_dev, lam_dev, E, nu_bg, nu_ref,
                                first, L0, err, s) != cudaSuccess)
        return MRF_ECUDA;
    if (cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MRF_ECUDA;
    return h_err ? MRF_EINVAL : MRF_OK;   // max_ray_len below the longest ray
}

size_t mrf_voxel_reduce_workspace(int64_t n_edges) {
    const int64_t nt = ceil_div(n_edges > 0 ? n_edges : 1, kTile);
    return (size_t)nt * (8 + 4 + 4 + 4) + 64;
}

int mrf_voxel_reduce(const uint32_t *perm_dev, const uint32_t *seg_off_dev, const uint32_t *seg_vox_dev,
                     int64_t n_seg, int64_t n_edges, const float *lam_dev, float logit_prior, float *T_dev,
                     void *workspace_dev, size_t workspace_bytes, void *stream) {
    if (n_edges < 0 || n_seg < 0) return MRF_EINVAL;
    if (n_edges >= ((int64_t)1 << 32)) return MRF_ERANGE;
    if (n_edges == 0) return MRF_OK;
    if (n_seg == 0 || !perm_dev || !seg_off_dev || !seg_vox_dev || !lam_dev || !T_dev || !workspace_dev)
        return MRF_EINVAL;
    if (workspace_bytes < mrf_voxel_reduce_workspace(n_edges)) return MRF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nt = ceil_div(n_edges, kTile);
    char *w = (char *)workspace_dev;
    uint32_t *plan = (uint32_t *)w;
    float *head = (float *)(w + nt * 8);
    float *tail = (float *)(w + nt * 12);
    uint32_t *tseg = (uint32_t *)(w + nt * 16);
    if (launch_reduce_plan(seg_off_dev, n_seg, n_edges, plan, nt, s) != cudaSuccess) return MRF_ECUDA;
    if (launch_voxel_reduce_f32(perm_dev, seg_off_dev, seg_vox_dev, plan, nt, lam_dev, T_dev, logit_prior, n_edges,
                                head, tail, tseg, s) != cudaSuccess)
        return MRF_ECUDA;
    return MRF_OK;
}


int mrf_add_heldout(mrf_ctx *c, const float *depth_dev, int32_t W, int32_t H, const double cam_to_world[12],
                    const mrf_intrinsics *K, const mrf_noise_lut *lut) {
    TRY(check_ctx(c));
    const int64_t npix = (int64_t)W * H;
    TravParams P;
    static thread_local TravTables TT;
    if (c->scenes.size() > 1) return fail(c, MRF_ESTATE, "held-out frames need a single-scene context");
    TRY(trav_params(c, 0, depth_dev, W, H, cam_to_world, K, lut, P, TT));
    Prof prof(c, K_TRAV);
    if (c->hR + npix + 1 > c->h_capR) {
        int64_t nc = c->h_capR + c->h_capR / 2;
        if (nc < c->hR + npix + 1) nc = c->hR + npix + 1;
        TRY(ensure(c, c->h_ray_off, (size_t)(nc + 1) * 8, true));
        TRY(ensure(c, c->h_Zr, (size_t)nc * 4, true));
        c->h_capR = nc;
    }
    TRY(ensure(c, c->counts, (size_t)npix * 4, false));
    TRY(ensure(c, c->rsetup, (size_t)npix * kRaySetupBytes, false));
    TRY(ensure(c, c->scan_ws, scan_workspace_bytes(npix), false));
    CUDA_TRY(c, cudaMemsetAsync(c->maxlen_dev.p, 0, 4, c->stream));
    CUDA_TRY(c, launch_ray_setup(P, TT, depth_dev, ptr<int32_t>(c->counts), ptr<float>(c->h_Zr) + c->hR,
                                 ptr<int32_t>(c->maxlen_dev), c->rsetup.p, c->stream));
    CUDA_TRY(c, exclusive_scan_i32_i64(ptr<int32_t>(c->counts), ptr<int64_t>(c->h_ray_off) + c->hR, npix, c->hE,
                                       c->scan_ws.p, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<int64_t>(c->h_ray_off) + c->hR + npix, 8, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t newE = c->h_pinned[0];
    if (newE >= ((int64_t)1 << 32) - kPad)
        return fail(c, MRF_ERANGE, "%lld held-out edges exceed the 2^32 edge limit", (long long)newE);
    if (newE + 1 > c->h_capE) {
        int64_t nc = c->h_capE + c->h_capE / 2;
        if (nc < newE + 1) nc = newE + 1;
        TRY(ensure(c, c->h_vox, (size_t)nc * 4, true));
        TRY(ensure(c, c->h_dmid, (size_t)nc * 4, true));
        c->h_capE = nc;
    }
    CUDA_TRY(c, launch_ray_walk(P, TT, c->rsetup.p, ptr<int64_t>(c->h_ray_off) + c->hR, ptr<uint32_t>(c->h_vox),
                                ptr<float>(c->h_dmid), nullptr, nullptr, nullptr, c->stream));
    c->launches += 5;
    c->hR += npix;
    c->hE = newE;
    return MRF_OK;
}

int mrf_accuracy(mrf_ctx *c, const float *depth_dev, int32_t W, int32_t H, const double cam_to_world[12],
                 const mrf_intrinsics *K, const mrf_noise_lut *lut, int8_t *result_dev, int64_t *n_accurate,
                 int64_t *n_evaluated) {
    TRY(check_ctx(c));
    if (!n_accurate || !n_evaluated) return fail(c, MRF_EINVAL, "null output");
    if (c->scenes.size() > 1) return fail(c, MRF_ESTATE, "the accuracy metric needs a single-scene context");
    const bool f64 = c->opt.precision == MRF_PREC_F64;
    if (f64 ? !c->T64.p : !c->T.p) return fail(c, MRF_ESTATE, "accuracy before infer");
    const int64_t npix = (int64_t)W * H;
    TravParams P;
    static thread_local TravTables TT;
    TRY(trav_params(c, 0, depth_dev, W, H, cam_to_world, K, lut, P, TT));
    P.no_trunc = 1;
    Prof prof(c, K_OTHER);
    TRY(ensure(c, c->ac_ray_off, (size_t)(npix + 1) * 8, false));
    TRY(ensure(c, c->ac_Z, (size_t)npix * 4, false));
    TRY(ensure(c, c->ac_cnt, 16, false));
    TRY(ensure(c, c->counts, (size_t)npix * 4, false));
    TRY(ensure(c, c->rsetup, (size_t)npix * kRaySetupBytes, false));
    TRY(ensure(c, c->scan_ws, scan_workspace_bytes(npix), false));
    CUDA_TRY(c, cudaMemsetAsync(c->maxlen_dev.p, 0, 4, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->ac_cnt.p, 0, 16, c->stream));
    CUDA_TRY(c, launch_ray_setup(P, TT, depth_dev, ptr<int32_t>(c->counts), ptr<float>(c->ac_Z),
                                 ptr<int32_t>(c->maxlen_dev), c->rsetup.p, c->stream));
    CUDA_TRY(c, exclusive_scan_i32_i64(ptr<int32_t>(c->counts), ptr<int64_t>(c->ac_ray_off), npix, 0, c->scan_ws.p,
                                       c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, ptr<int64_t>(c->ac_ray_off) + npix, 8, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t E = c->h_pinned[0];
    TRY(ensure(c, c->ac_vox, (size_t)(E + 1) * 4, false));
    TRY(ensure(c, c->ac_tin, (size_t)(E + 1) * 4, false));
    TRY(ensure(c, c->ac_tout, (size_t)(E + 1) * 4, false));
    CUDA_TRY(c, launch_ray_walk_seg(P, TT, c->rsetup.p, ptr<int64_t>(c->ac_ray_off), ptr<uint32_t>(c->ac_vox),
                                    ptr<float>(c->ac_tin), ptr<float>(c->ac_tout), c->stream));
    if (f64)
        CUDA_TRY(c, launch_omega(ptr<int64_t>(c->ac_ray_off), npix, ptr<uint32_t>(c->ac_vox), ptr<float>(c->ac_tin),
                                 ptr<float>(c->ac_tout), ptr<float>(c->ac_Z), ptr<double>(c->T64), (double)P.h,
                                 result_dev, ptr<unsigned long long>(c->ac_cnt), c->stream));
    else
        CUDA_TRY(c, launch_omega(ptr<int64_t>(c->ac_ray_off), npix, ptr<uint32_t>(c->ac_vox), ptr<float>(c->ac_tin),
                                 ptr<float>(c->ac_tout), ptr<float>(c->ac_Z), ptr<float>(c->T), (double)P.h,
                                 result_dev, ptr<unsigned long long>(c->ac_cnt), c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned, c->ac_cnt.p, 16, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *n_accurate = c->h_pinned[0];
    *n_evaluated = c->h_pinned[1];
    c->launches += 6;
    return MRF_OK;
}

int mrf_grad(mrf_ctx *c, int32_t iters, const mrf_noise_lut *theta, double *loss, double *grad_log_sigma,
             double *grad_outlier_w) {
    TRY(check_ctx(c));
    if (!theta || !theta->log_sigma || !loss || !grad_log_sigma || !grad_outlier_w)
        return fail(c, MRF_EINVAL, "null argument");
    if (iters < 0) return fail(c, MRF_EINVAL, "iters = %d", iters);
    if (theta->n_bins < 2 || theta->n_bins > kMaxBins || !(theta->d_hi > theta->d_lo) ||
        !(theta->outlier_w >= 0.f && theta->outlier_w < 1.f))
        return fail(c, MRF_EINVAL, "noise table out of range");
    if (c->opt.precision != MRF_PREC_F32) return fail(c, MRF_ESTATE, "mrf_grad needs an FP32 context");
    if (c->opt.variants) return fail(c, MRF_ESTATE, "the gradient is that of exact BP (no variants)");
    if (c->hR == 0 || c->hE == 0) return fail(c, MRF_ESTATE, "no held-out rays (mrf_add_heldout)");
    if (c->E == 0) return fail(c, MRF_ESTATE, "no frames");
    // theta as the likelihood of every edge
    static thread_local ThetaTab th;
    th.n_bins = theta->n_bins;
    th.has_bias = theta->bias != nullptr;
    th.dlo = theta->d_lo;
    th.dhi = theta->d_hi;
    th.delta = ((double)theta->d_hi - (double)theta->d_lo) / theta->n_bins;
    th.w = theta->outlier_w;
    for (int k = 0; k < theta->n_bins; ++k) {
        th.ls[k] = theta->log_sigma[k];
        th.bias[k] = theta->bias ? theta->bias[k] : 0.f;
    }
    theta_far_setup(th);
    const double floor_d = th.w / th.dhi;
    const bool bg_from_w = c->opt.nu_bg < 0.f;
    c->nu_bg = bg_from_w ? floor_d : (double)c->opt.nu_bg;
    c->nu_floor = (float)floor_d;
    CUDA_TRY(c, launch_nu_theta(th, ptr<int64_t>(c->ray_off), c->R, ptr<float>(c->dmid), ptr<float>(c->Zr),
                                ptr<float>(c->nu), c->stream));
    c->launches += 1;
    TRY(ensure_edge_transpose(c));   // the reverse pass sums per voxel over edges
    const int64_t E = c->E, Vk = c->Vk, K = iters, R = c->R, hR = c->hR, hE = c->hE;
    // forward, keeping every pass
    TRY(ensure(c, c->gr_ck_lam, (size_t)(K > 0 ? K : 1) * E * 4, false));
    TRY(ensure(c, c->gr_ck_T, (size_t)(K > 0 ? K : 1) * Vk * 4, false));
    TRY(infer_impl(c, iters, ptr<float>(c->gr_ck_lam), ptr<float>(c->gr_ck_T)));
    const float *TK = ptr<float>(c->T);
    // held-out loss and d loss / d T^K
    TRY(ensure(c, c->gr_hQ, (size_t)hE * 8, false));
    TRY(ensure(c, c->gr_hnu, (size_t)hE * 8, false));
    TRY(ensure(c, c->gr_hgp, (size_t)(hE + kPad) * 8, false));
    TRY(ensure(c, c->gr_hgnu, (size_t)hE * 8, false));
    TRY(ensure(c, c->gr_hloss, (size_t)hR * 8, false));
    TRY(ensure(c, c->gr_hgbg, (size_t)hR * 8, false));
    TRY(ensure(c, c->gr_gT, (size_t)Vk * 8, false));
    CUDA_TRY(c, launch_heldout(th, ptr<int64_t>(c->h_ray_off), hR, ptr<uint32_t>(c->h_vox), ptr<float>(c->h_dmid),
                               ptr<float>(c->h_Zr), TK, c->nu_bg, ptr<double>(c->gr_hQ), ptr<double>(c->gr_hnu),
                               ptr<double>(c->gr_hgp), ptr<double>(c->gr_hgnu), ptr<double>(c->gr_hloss),
                               ptr<double>(c->gr_hgbg), c->stream));
    int64_t hS = 0, hnt = 0;
    TRY(edge_transpose(c, ptr<uint32_t>(c->h_vox), hE, c->gr_hperm, c->gr_hso, c->gr_hsv, c->gr_hplan, &hS, &hnt));
    const int64_t ntr = c->n_red_tiles > hnt ? c->n_red_tiles : hnt;
    TRY(ensure(c, c->gr_head, (size_t)ntr * 8, false));
    TRY(ensure(c, c->gr_tail, (size_t)ntr * 8, false));
    TRY(ensure(c, c->gr_tseg, (size_t)ntr * 4, false));
    CUDA_TRY(c, cudaMemsetAsync(c->gr_gT.p, 0, (size_t)Vk * 8, c->stream));
    CUDA_TRY(c, launch_voxel_reduce_f64(ptr<uint32_t>(c->gr_hperm), ptr<uint32_t>(c->gr_hso),
                                        ptr<uint32_t>(c->gr_hsv), ptr<uint32_t>(c->gr_hplan), hnt,
                                        ptr<double>(c->gr_hgp), ptr<double>(c->gr_gT), 0.0, hE,
                                        ptr<double>(c->gr_head), ptr<double>(c->gr_tail),
                                        ptr<uint32_t>(c->gr_tseg), c->stream));
    CUDA_TRY(c, launch_sigmoid_adjoint(TK, ptr<double>(c->gr_gT), Vk, c->stream));
    c->launches += 4;
    // the passes, last to first
    const double gamma = c->prior;
    const double ip = c->opt.init_p > 0.f ? (double)c->opt.init_p : gamma;
    const float L0 = (float)(log(ip) - log1p(-ip));
    const float nu_bg_f = (float)c->nu_bg;   // the values the FP32 messages used
    const float nu_ref = fminf(nu_bg_f, c->nu_floor);
    for (Buf *b : {&c->gr_glam, &c->gr_gL, &c->gr_gLn, &c->gr_sP, &c->gr_sA, &c->gr_sB, &c->gr_sg})
        TRY(ensure(c, *b, (size_t)(E + kPad) * 8, false));
    TRY(ensure(c, c->gr_gnu, (size_t)E * 8, false));
    TRY(ensure(c, c->gr_gbg, (size_t)R * 8, false));
    CUDA_TRY(c, cudaMemsetAsync(c->gr_gLn.p, 0, (size_t)E * 8, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->gr_gnu.p, 0, (size_t)E * 8, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->gr_gbg.p, 0, (size_t)R * 8, c->stream));
    for (int64_t t = K; t >= 1; --t) {
        CUDA_TRY(c, launch_glam(ptr<double>(c->gr_gT), ptr<uint32_t>(c->vox), ptr<double>(c->gr_gLn), E,
                                ptr<double>(c->gr_glam), c->stream));
        const float *Tprev = t >= 2 ? ptr<float>(c->gr_ck_T) + (size_t)(t - 2) * Vk : nullptr;
        const float *lprev = t >= 2 ? ptr<float>(c->gr_ck_lam) + (size_t)(t - 2) * E : nullptr;
        CUDA_TRY(c, launch_ray_adjoint(ptr<int64_t>(c->ray_off), R, ptr<uint32_t>(c->vox), ptr<float>(c->nu), Tprev,
                                       lprev, L0, t == 1, nu_bg_f, nu_ref, ptr<double>(c->gr_glam),
                                       ptr<float>(c->gr_sP) + (E + kPad), ptr<float>(c->gr_sP),
                                       ptr<float>(c->gr_sA), ptr<float>(c->gr_sB),
                                       ptr<float>(c->gr_sg), ptr<double>(c->gr_gL), ptr<double>(c->gr_gnu),
                                       ptr<double>(c->gr_gbg), c->stream));
        c->launches += 2;
        if (t >= 2) {
            CUDA_TRY(c, cudaMemsetAsync(c->gr_gT.p, 0, (size_t)Vk * 8, c->stream));
            CUDA_TRY(c, launch_voxel_reduce_f64(ptr<uint32_t>(c->perm), ptr<uint32_t>(c->seg_off),
                                                ptr<uint32_t>(c->seg_vox), ptr<uint32_t>(c->red_plan),
                                                c->n_red_tiles, ptr<double>(c->gr_gL), ptr<double>(c->gr_gT), 0.0, E,
                                                ptr<double>(c->gr_head), ptr<double>(c->gr_tail),
                                                ptr<uint32_t>(c->gr_tseg), c->stream));
            c->launches += 2;
        }
        std::swap(c->gr_gL, c->gr_gLn);
    }
    // the table: through every training and held-out edge's nu, and nu_bg
    const int nb = th.n_bins + 1;
    const int tpb = theta_grad_threads(th.n_bins);
    const int blk_tr = (int)(ceil_div(R, tpb) < 1024 ? ceil_div(R, tpb) : 1024);
    const int blk_ho = (int)(ceil_div(hR, tpb) < 1024 ? ceil_div(hR, tpb) : 1024);
    TRY(ensure(c, c->gr_part, (size_t)(blk_tr + blk_ho) * nb * 8, false));
    CUDA_TRY(c, launch_theta_grad(th, ptr<int64_t>(c->ray_off), R, ptr<float>(c->dmid), ptr<float>(c->Zr),
                                  ptr<double>(c->gr_gnu), ptr<double>(c->gr_part), blk_tr, c->stream));
    CUDA_TRY(c, launch_theta_grad(th, ptr<int64_t>(c->h_ray_off), hR, ptr<float>(c->h_dmid), ptr<float>(c->h_Zr),
                                  ptr<double>(c->gr_hgnu), ptr<double>(c->gr_part) + (size_t)blk_tr * nb, blk_ho,
                                  c->stream));
    c->launches += 2;
    std::vector<double> part((size_t)(blk_tr + blk_ho) * nb), hl((size_t)hR), gb((size_t)R), hgb((size_t)hR);
    CUDA_TRY(c, cudaMemcpyAsync(part.data(), c->gr_part.p, part.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(hl.data(), c->gr_hloss.p, hl.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(gb.data(), c->gr_gbg.p, gb.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(hgb.data(), c->gr_hgbg.p, hgb.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    TRY(device_errors(c));
    double L = 0.0, gbg = 0.0;
    for (double x : hl) L += x;
    for (double x : gb) gbg += x;
    for (double x : hgb) gbg += x;
    for (int k = 0; k < nb; ++k) {
        double s = 0.0;
        for (int b = 0; b < blk_tr + blk_ho; ++b) s += part[(size_t)b * nb + k];
        if (k < th.n_bins) grad_log_sigma[k] = s;
        else *grad_outlier_w = s + (bg_from_w ? gbg / th.dhi : 0.0);
    }
    *loss = L;
    return MRF_OK;
}

int mrf_set_plan(mrf_ctx *c, int32_t ray_items, int32_t threads, int32_t groups) {
    TRY(check_ctx(c));
    if (!(ray_items == 0 || ray_items == 4 || ray_items == 8 || ray_items == 16 || ray_items == 32))
        return fail(c, MRF_EINVAL, "ray_items %d", ray_items);
    if (!(threads == 0 || threads == -1 || threads == 128 || threads == kThreads || threads == 512))
        return fail(c, MRF_EINVAL, "threads %d", threads);
    if (!(groups >= -1 && groups <= 1)) return fail(c, MRF_EINVAL, "groups %d", groups);
    c->plan_items = ray_items;
    c->plan_threads = threads;
    c->plan_groups = groups;
    c->dirty = true;
    return MRF_OK;
}

int mrf_infer_graph(mrf_ctx *c, int32_t iters) {
    TRY(check_ctx(c));
    if (iters < 0) return fail(c, MRF_EINVAL, "iters = %d", iters);
    if (c->dirty) TRY(build_transpose(c));
    if (!c->gstream) {
        CUDA_TRY(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        for (auto &e : c->gev) CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (!c->graph || c->graph_iters != iters) {
        if (c->graph) cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        // an ordinary run first: it makes every allocation and kernel set-up,
        // and its result is this call's
        TRY(infer_impl(c, iters));
        const int64_t l0 = c->launches;
        CUDA_TRY(c, cudaEventRecord(c->gev[0], c->stream));
        CUDA_TRY(c, cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
        cudaStream_t user = c->stream;
        c->stream = c->gstream;
        c->capturing = true;
        cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? infer_impl(c, iters) : MRF_ECUDA;
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
        c->capturing = false;
        c->stream = user;
        if (rc == MRF_OK && (e != cudaSuccess || e2 != cudaSuccess || !g))
            rc = fail(c, MRF_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        if (rc == MRF_OK) {
            e = cudaGraphInstantiate(&c->graph, g, 0);
            if (e != cudaSuccess) rc = fail(c, MRF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        if (g) cudaGraphDestroy(g);
        if (rc != MRF_OK) {
            c->graph = nullptr;
            return rc;
        }
        c->graph_iters = iters;
        c->graph_launches = c->launches - l0;
        c->launches = l0;
        return MRF_OK;
    }
    // replay, ordered after earlier work on the context's stream and before later work
    CUDA_TRY(c, cudaEventRecord(c->gev[0], c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    CUDA_TRY(c, cudaGraphLaunch(c->graph, c->gstream));
    CUDA_TRY(c, cudaEventRecord(c->gev[1], c->gstream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->gev[1], 0));
    c->launches += c->graph_launches;
    return MRF_OK;
}
}  // extern "C"
