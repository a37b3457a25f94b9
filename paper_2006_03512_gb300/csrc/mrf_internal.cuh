// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/mrfmap.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace mrf {

// ---------------------------------------------------------------- constants
constexpr int kThreads = 256;          // every kernel in this library uses 256-thread CTAs
constexpr int kItems = 16;             // items per thread for scans, sort and voxel reduction
constexpr int kTile = kThreads * kItems;
constexpr int kMaxBins = 512;          // sensor-noise table entries accepted by the traversal
constexpr float kLamClamp = 64.f;      // |log-odds message| bound (one-voxel rays with nu_bg = 0)
constexpr uint32_t kNone = 0xffffffffu;

// ---------------------------------------------------------------- voxel keys
// Internal voxel key: the grid is cut into 8x8x8 bricks, numbered x-fastest, and
// the 512 voxels of a brick are numbered in Morton (z-) order, so voxels close
// in space get close keys.  A ray's consecutive voxels then share cache lines,
// and a run of voxel-sorted edges covers a compact block of space.
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {  // bits 0,1,2 -> 0,3,6
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t m) {  // bits 0,3,6 -> 0,1,2
    return (m & 1u) | ((m >> 2) & 2u) | ((m >> 4) & 4u);
}
__host__ __device__ __forceinline__ uint32_t voxel_key(uint32_t x, uint32_t y, uint32_t z, uint32_t nbx,
                                                       uint32_t nby) {
    const uint32_t b = (x >> 3) + nbx * ((y >> 3) + nby * (z >> 3));
    return (b << 9) | spread3(x & 7u) | (spread3(y & 7u) << 1) | (spread3(z & 7u) << 2);
}
__host__ __device__ __forceinline__ void key_xyz(uint32_t key, uint32_t nbx, uint32_t nby, uint32_t &x,
                                                 uint32_t &y, uint32_t &z) {
    const uint32_t b = key >> 9, m = key & 511u;
    x = ((b % nbx) << 3) | compact3(m);
    y = (((b / nbx) % nby) << 3) | compact3(m >> 1);
    z = ((b / (nbx * nby)) << 3) | compact3(m >> 2);
}

// ----------------------------------------------------------- traversal args
// Per-frame constants, computed on the host exactly as the pinned recipe says
// (camera centre in voxel units and rotation rounded from double to float).
struct TravParams {
    int nx, ny, nz;
    uint32_t nbx, nby;    // bricks along x and y (voxel keys)
    uint32_t key_base;    // first key of the frame's scene (batched contexts)
    int no_trunc;         // walk to the grid exit (the evaluation metric), not 3 sigma past Z
    float h;              // voxel edge (metres)
    float o[3];           // camera centre in voxel units
    float R[9];           // camera-to-world rotation, row-major, float
    float fx, fy, cx, cy;
    int W, H;
    int n_bins;
    float dlo, inv_delta; // table bin rule in float: x = (d - dlo) * inv_delta - 0.5
    float w1, w_floor;    // 1 - outlier_w, outlier_w / d_hi
    double dlo_d, delta_d, w_d, floor_d;  // FP64 versions for the FP64 path
    int has_bias;
    int far_ok;           // the far-edge test below may replace the FP64 likelihood
};

struct TravTables {
    float log_sigma[kMaxBins];
    float sig[kMaxBins];   // (float)exp((double)log_sigma[k]) -- the truncation table
    float bias[kMaxBins];
    // Far edges: for an edge whose FP32 bin is k, 0.5 (|Z - d| far_inv_sig[k])^2
    // > far_thr[k] guarantees (1 - w) N(Z; d, sigma(d)) < w / d_hi * 2^-30, so
    // the likelihood rounds to the float of its floor (bins k-1 .. k+2 bound
    // sigma, which covers an FP32 bin off by one; built on the host).
    float far_inv_sig[kMaxBins];
    float far_thr[kMaxBins];
};

// ------------------------------------------------------------------ launches
// traverse.cu
// setup: kRaySetupBytes per pixel, written by the set-up and read by the walk
constexpr int kRaySetupBytes = 64;
cudaError_t launch_ray_setup(const TravParams &P, const TravTables &TT, const float *depth, int32_t *counts,
                             float *Zr, int32_t *max_len, void *setup, cudaStream_t s);
cudaError_t launch_ray_walk(const TravParams &P, const TravTables &TT, const void *setup, const int64_t *ray_off,
                            uint32_t *vox, float *dmid, float *nu, double *nu64, float *wlen, cudaStream_t s);
// the walk with each voxel's entry and exit range (no midpoints, no likelihoods)
cudaError_t launch_ray_walk_seg(const TravParams &P, const TravTables &TT, const void *setup, const int64_t *ray_off,
                                uint32_t *vox, float *t_in, float *t_out, cudaStream_t s);

// scan.cu : out[0..n] = base + exclusive prefix sums of in[0..n-1] (out[n] = base + total)
size_t scan_workspace_bytes(int64_t n);
cudaError_t exclusive_scan_i32_i64(const int32_t *in, int64_t *out, int64_t n, int64_t base, void *ws,
                                   cudaStream_t s);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, void *ws, cudaStream_t s);

// sort.cu : stable LSD radix sort of (key, edge id) pairs and the segment list
size_t sort_workspace_bytes(int64_t n);
cudaError_t radix_sort_edges(const uint32_t *keys_in, int key_bits, int64_t n, uint32_t *keys_a,
                             uint32_t *keys_b, uint32_t *vals_tmp, uint32_t *vals_out, uint32_t **keys_sorted,
                             void *ws, cudaStream_t s, int64_t *n_launches);
cudaError_t segment_heads(const uint32_t *sorted_keys, int64_t n, uint32_t *flags, cudaStream_t s);
cudaError_t segment_emit(const uint32_t *sorted_keys, const uint32_t *head_idx, int64_t n, uint32_t *seg_off,
                         uint32_t *seg_vox, cudaStream_t s);

// bp.cu
int ray_tile_items(int32_t max_len);   // 8, 16 or 32 items per thread; 0 if the ray is too long
int64_t ray_tile_window(int kt, int32_t max_len);
cudaError_t launch_ray_plan(const int64_t *ray_off, int64_t R, int64_t E, int64_t window, uint32_t *tile_r0,
                            int64_t ntiles, cudaStream_t s);
cudaError_t launch_ray_messages_f32(int kt, const int64_t *ray_off, const uint32_t *tile_r0, int64_t ntiles,
                                    const uint32_t *vox, const float *nu, const float *T, float *lam,
                                    int64_t n_alloc, float nu_bg, float nu_ref, int first, float L0, uint32_t *err,
                                    cudaStream_t s, const float *wlen = nullptr);
// group.cu : group tables, one CTA per tile (cap = the tile's window, 2048 or 4096; hb = ray starts)
cudaError_t launch_tile_sort(int cap, const int64_t *tile_E, int64_t ntiles, const uint32_t *hb, const uint32_t *vox,
                             uint16_t *lidx, uint32_t *ends, uint16_t *gid, int32_t *gcount, uint32_t *gtmp,
                             cudaStream_t s);
// the group keys by slot, from the tile-groups kernel's per-tile copies in gtmp
cudaError_t launch_group_keys(const int64_t *tile_E, int64_t ntiles, const int64_t *tg_off, const uint32_t *gtmp,
                              uint32_t *gkey, cudaStream_t s);
// group.cu : (keyframe, voxel) pairs over the voxel-major edge order, and the
// per-pair average of the stored messages
cudaError_t launch_pair_flags(const uint32_t *perm, const uint32_t *vox, int64_t E, const int64_t *frame_E,
                              int32_t n_frames, int32_t *flags, cudaStream_t s);
cudaError_t launch_pair_starts(const int32_t *flags, const int64_t *pos, int64_t E, uint32_t *pair_off,
                               uint32_t *pid, uint32_t *ident, cudaStream_t s);
cudaError_t launch_pair_scatter(const uint32_t *perm, const uint32_t *pid, const uint32_t *pair_off,
                                const float *sums, int64_t E, float *lam, cudaStream_t s);
// ray_pipe.cu : persistent TMA-pipelined ray kernel on the context's padded arrays
bool ray_pipe_supported(int kt, int nt);
// whole rays packed greedily into tiles of at most cap edges, restarting every
// chunk of rays: counts per chunk (tile_off null), then the tiles' first edges
// at tile_E + tile_off[chunk]
int64_t tile_pack_chunks(int64_t R);
cudaError_t launch_tile_pack(const int64_t *ray_off, int64_t R, int64_t cap, int32_t *counts, const int64_t *tile_off,
                             int64_t *tile_E, cudaStream_t s);
cudaError_t launch_ray_pipe_plan(const int64_t *ray_off, int64_t R, const uint32_t *tile_r0, int64_t ntiles,
                                 int64_t *tile_E, uint32_t *hb, int64_t hb_words, cudaStream_t s);
cudaError_t launch_ray_pipe(int kt, int nt, bool bf16, int64_t n_sm, const int64_t *tile_E, int64_t ntiles,
                            const uint32_t *hb, const uint32_t *vox, const float *nu, const float *T, void *lam,
                            float nu_bg, float nu_ref, int first, float L0, uint32_t *err, const uint16_t *lidx,
                            const uint32_t *ends, const uint16_t *gid, const uint32_t *gkey, const int64_t *tg_off,
                            float *partial, cudaStream_t s, bool floored = false);
// a bounded wait that times out (nothing arrives): sets bit 4 of err after ~1 s
cudaError_t launch_wait_probe(uint32_t *err, cudaStream_t s);
// bf16 messages (raw 16-bit patterns) -> FP32, exactly
cudaError_t launch_bf16_to_f32(const void *in, float *out, int64_t n, cudaStream_t s);
cudaError_t launch_reduce_plan(const uint32_t *seg_off, int64_t n_seg, int64_t E, uint32_t *plan,
                               int64_t ntiles, cudaStream_t s);
cudaError_t launch_voxel_reduce_f32(const uint32_t *perm, const uint32_t *seg_off, const uint32_t *seg_vox,
                                    const uint32_t *plan, int64_t ntiles, const float *lam, float *T,
                                    float logit_prior, int64_t E, float *head_part, float *tail_part,
                                    uint32_t *tail_seg, cudaStream_t s);
cudaError_t launch_voxel_reduce_f64(const uint32_t *perm, const uint32_t *seg_off, const uint32_t *seg_vox,
                                    const uint32_t *plan, int64_t ntiles, const double *lam, double *T,
                                    double logit_prior, int64_t E, double *head_part, double *tail_part,
                                    uint32_t *tail_seg, cudaStream_t s);
// bp.cu : the messages of listed long rays with FP64 accumulations (FP32 context), and their scatter
cudaError_t launch_long_rays_f64(const int64_t *ray_off, const uint32_t *ids, int64_t n_long, const int64_t *loff,
                                 const uint32_t *vox, const float *nu, const float *T, const float *lam, int first,
                                 double L0, double nu_bg, float *out, double *bscr, cudaStream_t s);
cudaError_t launch_long_scatter(const int64_t *ray_off, const uint32_t *ids, int64_t n_long, const int64_t *loff,
                                const float *out, float *lam, cudaStream_t s);
// the paper's log-domain form in FP32 (an ablation; lbscr: E floats of scratch)
cudaError_t launch_ray_messages_log32(const int64_t *ray_off, int64_t R, const uint32_t *vox, const float *nu,
                                      const float *T, float *lam, float *lbscr, float nu_bg, int first, float L0,
                                      cudaStream_t s);
cudaError_t launch_ray_messages_f64(const int64_t *ray_off, int64_t R, const uint32_t *vox, const double *nu,
                                    const double *T, double *lam, double *bscratch, double nu_bg, int first,
                                    double L0, cudaStream_t s);
cudaError_t launch_fill_f32(float *p, int64_t n, float v, cudaStream_t s);
cudaError_t launch_fill_f64(double *p, int64_t n, double v, cudaStream_t s);
struct GridMap {   // linear x-fastest index <-> internal voxel key
    uint32_t nx, ny, nz, nbx, nby;
};
cudaError_t launch_marginals_f32(const float *T, float *p, GridMap gm, cudaStream_t s);
cudaError_t launch_marginals_f64(const double *T, float *p, GridMap gm, cudaStream_t s);
cudaError_t launch_gather_linear_f32(const float *T, float *out, GridMap gm, cudaStream_t s);
cudaError_t launch_gather_linear_f64(const double *T, double *out, GridMap gm, cudaStream_t s);
cudaError_t launch_keys_to_linear(const uint32_t *keys, uint32_t *out, int64_t n, GridMap gm, cudaStream_t s);
cudaError_t launch_f64_to_f32(const double *a, float *b, int64_t n, cudaStream_t s);

// noise table as the gradient's variable: FP64 log sigma at the bin centres
// and outlier weight (grad.cu)
struct ThetaTab {
    int n_bins, has_bias;
    double dlo, delta, dhi, w;
    double ls[kMaxBins];
    float bias[kMaxBins];
    // Far edges (set on the host by theta_far_setup): an edge whose FP32 table
    // bin is k and |Z - d| > far_d[k] has (1 - w) N(Z; d + b, sigma) below 2^-40
    // of the likelihood floor (bins k-1 .. k+1 bound sigma and b), so its
    // likelihood rounds to nu_far (the floor's float) and its partials are
    // d nu / d log sigma = 0, d nu / d w = 1 / d_hi to that relative accuracy.
    // far_ok = 0 (the floor's double too close to a float rounding boundary)
    // sends every edge through the exact evaluation.
    int far_ok;
    float dlo_f, inv_delta_f, nu_far;
    float far_d[kMaxBins];
};
// fills the far-edge fields of th from its table (host)
void theta_far_setup(ThetaTab &th);
cudaError_t launch_nu_theta(const ThetaTab &th, const int64_t *ray_off, int64_t R, const float *dmid,
                            const float *Zr, float *nu, cudaStream_t s);
cudaError_t launch_heldout(const ThetaTab &th, const int64_t *ray_off, int64_t R, const uint32_t *vox,
                           const float *dmid, const float *Zr, const float *T, double nu_bg, double *Q, double *nuh,
                           double *gp, double *gnu, double *loss_r, double *gbg, cudaStream_t s);
cudaError_t launch_sigmoid_adjoint(const float *T, double *g, int64_t V, cudaStream_t s);
cudaError_t launch_glam(const double *gT, const uint32_t *vox, const double *gLn, int64_t E, double *glam,
                        cudaStream_t s);
cudaError_t launch_ray_adjoint(const int64_t *ray_off, int64_t R, const uint32_t *vox, const float *nu,
                               const float *Tprev, const float *lprev, float L0, int first, float nu_bg,
                               float nu_ref, const double *glam, float *sL, float *sP, float *sA, float *sB,
                               float *sD, double *gL, double *gnu, double *gbg, cudaStream_t s);
int theta_grad_threads(int n_bins);
cudaError_t launch_theta_grad(const ThetaTab &th, const int64_t *ray_off, int64_t R, const float *dmid,
                              const float *Zr, const double *gnu, double *part, int blocks, cudaStream_t s);

// the evaluation metric (grad.cu): one thread per ray walked to the grid exit
template <class V>
cudaError_t launch_omega(const int64_t *ray_off, int64_t R, const uint32_t *vox, const float *t_in,
                         const float *t_out, const float *Zr, const V *T, double h, int8_t *result,
                         unsigned long long *counts, cudaStream_t s);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace mrf
