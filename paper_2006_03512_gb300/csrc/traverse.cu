// Ray set-up and 3D-DDA traversal (Section IV-A; truncation of Section IV-B).
//
// This translation unit is compiled with -fmad=false and IEEE division and
// square root so that every FP32 operation below is one correctly rounded
// IEEE operation in the order written.  That makes the voxel sequence and the
// per-voxel midpoint ranges of every ray a pure function of the inputs, equal
// bit for bit to any other implementation of the same recipe.
//
// Recipe (per pixel (u, v) with z-depth z; o and R come rounded from double):
//   a = ((float)u - cx) / fx;  b = ((float)v - cy) / fy;  len = sqrt((a*a + b*b) + 1)
//   e_q = (R_q0 a + R_q1 b) + R_q2;  k_q = (e_q / len) / h  (voxels per metre)
//   Z = z * len  (measured range along the ray)
//   slab clip: t0 = max(0, lo_q), t_exit = min(hi_q) over axes with k_q != 0
//   t1 = min(t_exit, Z + 3 sigma_trunc(Z))   (sigma table interpolated in sigma)
//   start s_q = clamp(floor(o_q + t0 k_q)), end e_q = clamp(floor(o_q + t1 k_q)),
//   e forced onto the stepping side of s; N = 1 + sum |e_q - s_q|
//   step: among axes not yet at e, the smallest t of the next face
//   ((float)(c_q + [k_q > 0]) - o_q) * inv_q, ties to the lower axis;
//   segment t_out = max(t_in, min(t_face, t1)), last segment ends at t1;
//   recorded depth d = 0.5 (t_in + t_out) in metres; the voxel is stored by its
//   internal key (brick + Morton order), exported as x + nx (y + ny z).
#include <math.h>

#include "mrf_internal.cuh"

namespace mrf {
namespace {

// one ray's set-up, written by k_ray_setup and read by the walk (64 bytes)
struct alignas(16) RaySetup {
    float k[3], inv[3];
    float t0, t1, Z;
    int s[3], e[3];
    int N;
};
static_assert(sizeof(RaySetup) == 64, "four 16-byte words per ray");

__device__ __forceinline__ int clamp_floor(float x, int n) {
    float f = floorf(x);
    if (!(f >= 0.0f)) return 0;
    if (f > (float)(n - 1)) return n - 1;
    return (int)f;
}

__device__ __forceinline__ void bin_rule(const TravParams &P, float d, int &k, float &f) {
    float x = (d - P.dlo) * P.inv_delta - 0.5f;
    float fk = floorf(x);
    if (!(fk >= 0.0f)) k = 0;
    else if (fk > (float)(P.n_bins - 2)) k = P.n_bins - 2;
    else k = (int)fk;
    f = x - (float)k;
    if (f < 0.0f) f = 0.0f;
    if (f > 1.0f) f = 1.0f;
}

__device__ __forceinline__ float trunc_sigma(const TravParams &P, const TravTables &TT, float Z) {
    int k;
    float f;
    bin_rule(P, Z, k, f);
    float a = (1.0f - f) * TT.sig[k];
    float b = f * TT.sig[k + 1];
    return a + b;
}

__device__ __forceinline__ void ray_setup(const TravParams &P, const TravTables &TT, int u, int v, float z,
                                          RaySetup &r) {
    const int n[3] = {P.nx, P.ny, P.nz};
    const bool valid = (z > 0.0f) && isfinite(z);
    const float a = ((float)u - P.cx) / P.fx;
    const float b = ((float)v - P.cy) / P.fy;
    const float aa = a * a;
    const float bb = b * b;
    const float len = sqrtf((aa + bb) + 1.0f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float ea = P.R[q * 3 + 0] * a;
        const float eb = P.R[q * 3 + 1] * b;
        const float e = (ea + eb) + P.R[q * 3 + 2];
        r.k[q] = (e / len) / P.h;
    }
    r.Z = z * len;
    float t0 = 0.0f, tex = INFINITY;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (r.k[q] != 0.0f) {
            const float inv = 1.0f / r.k[q];
            const float ta = (0.0f - P.o[q]) * inv;
            const float tb = ((float)n[q] - P.o[q]) * inv;
            const float lo = ta < tb ? ta : tb;
            const float hi = ta < tb ? tb : ta;
            r.inv[q] = inv;
            if (lo > t0) t0 = lo;
            if (hi < tex) tex = hi;
        } else {
            r.inv[q] = 0.0f;
            if (!(P.o[q] >= 0.0f && P.o[q] < (float)n[q])) ok = false;
        }
    }
    const float sig = valid && !P.no_trunc ? trunc_sigma(P, TT, r.Z) : 0.0f;
    const float tt = r.Z + 3.0f * sig;
    const float t1 = P.no_trunc || tex < tt ? tex : tt;
    r.t0 = t0;
    r.t1 = t1;
    r.N = 0;
    if (!(valid && ok && t0 < t1)) return;
    int N = 1;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float ps = P.o[q] + t0 * r.k[q];
        const float pe = P.o[q] + t1 * r.k[q];
        const int s = clamp_floor(ps, n[q]);
        int e = clamp_floor(pe, n[q]);
        if (r.k[q] > 0.0f) {
            if (e < s) e = s;
        } else if (r.k[q] < 0.0f) {
            if (e > s) e = s;
        } else {
            e = s;
        }
        r.s[q] = s;
        r.e[q] = e;
        N += e > s ? e - s : s - e;
    }
    r.N = N;
}

// nu(d) = (1 - w) N(Z; d + b(d), sigma(d)) + w / d_hi with log sigma(d)
// interpolated from the table (Eq. "noise", Section IV-C).  Evaluated once per
// edge in FP64 (bin rule in double); the FP32 path stores it rounded to float.
// ls_tab / bias_tab: the table's log sigma and bias (shared-memory copies in the walk)
__device__ __forceinline__ double sensor_nu_f64(const TravParams &P, const float *ls_tab, const float *bias_tab,
                                                double d, double Z) {
    const double x = (d - P.dlo_d) / P.delta_d - 0.5;
    const double fk = floor(x);
    int k;
    if (!(fk >= 0.0)) k = 0;
    else if (fk > P.n_bins - 2) k = P.n_bins - 2;
    else k = (int)fk;
    double f = x - k;
    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
    const double ls = (1.0 - f) * (double)ls_tab[k] + f * (double)ls_tab[k + 1];
    const double b = P.has_bias ? (1.0 - f) * (double)bias_tab[k] + f * (double)bias_tab[k + 1] : 0.0;
    const double zz = (Z - (d + b)) * exp(-ls);
    const double lg = -0.5 * zz * zz - ls - 0.91893853320467274178;
    if (P.w_d <= 0.0) return exp(lg);
    return (1.0 - P.w_d) * exp(lg) + P.floor_d;
}

// true when the edge's likelihood is its floor to float precision (see TravTables)
__device__ __forceinline__ bool far_edge(const TravParams &P, const float *inv_sig, const float *thr, float d,
                                         float Z) {
    int k;
    float f;
    bin_rule(P, d, k, f);
    const float x = fabsf(Z - d) * inv_sig[k];
    return 0.5f * x * x > thr[k];
}

__global__ void __launch_bounds__(kThreads) k_ray_setup(const __grid_constant__ TravParams P,
                                                        const __grid_constant__ TravTables TT,
                                                        const float *__restrict__ depth, int32_t *__restrict__ counts,
                                                        float *__restrict__ Zr, int32_t *__restrict__ max_len,
                                                        RaySetup *__restrict__ setup) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = (int64_t)P.W * P.H;
    int N = 0;
    if (p < npix) {
        RaySetup r = {};
        ray_setup(P, TT, (int)(p % P.W), (int)(p / P.W), depth[p], r);
        N = r.N;
        counts[p] = N;
        Zr[p] = r.Z;
        setup[p] = r;
    }
    // warp max, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) N = max(N, __shfl_xor_sync(0xffffffffu, N, o));
    if ((threadIdx.x & 31) == 0 && N > 0) atomicMax(max_len, N);
}

// ---- the walk, one warp per ray.  The step rule above takes, among the axes
// not yet at their end cell, the smallest next-face time, ties to the lower
// axis.  Axis q's j-th face time,
//   T_q(j) = ((float)(s_q + dir_q j + [k_q > 0]) - o_q) * inv_q,
// depends on j alone and is non-decreasing in j (rounding is monotone), so
// the walk's steps are the stable merge of the three axes' face times by
// (time, axis).  Step j of axis q is therefore the merge's element number
//   rank = j + (faces of the other axes that come before it in that order),
// each count found from the continuous estimate floor(o + T k) and corrected
// with exact face times; the step enters edge rank + 1, whose cell is s moved
// by the counts and whose range is [max(t0, min(T, t1)), max(t0, min(M, t1))]
// with M the smallest of the three axes' next face times (t1 on the last
// edge).  These are the values the sequential walk computes, operation for
// operation, so every edge is produced bit for bit without the walk's
// dependent chain: a lane per step, coalesced within a ray.
//
// FP64 likelihoods near the measured range (a few edges per ray) go through a
// per-warp queue and are evaluated 32 at a time, so that the slow FP64 units
// run with every lane busy.
struct WalkAxis {
    int s, n, dir, base;   // start cell, steps, +-1, s + [k > 0]
    float o, k, inv;
};

// face time of step j of axis A
__device__ __forceinline__ float face_t(const WalkAxis &A, int j) {
    return ((float)(A.base + A.dir * j) - A.o) * A.inv;
}

// The number of steps of axis A that the merge puts before a step at time T
// (le: A is the lower axis, so equal times come before), and A's next face
// time after them (infinity when A is exhausted).  The loops move g
// monotonically within [0, n].
__device__ __forceinline__ int steps_before(const WalkAxis &A, float T, bool le, float &head) {
    int g = 0;
    if (A.n > 0) {
        const float p = A.o + T * A.k;
        const float fl = floorf(p);
        const float gf = A.dir > 0 ? fl - (float)A.s : (float)A.s - fl;
        g = !(gf > 0.0f) ? 0 : (gf >= (float)A.n ? A.n : (int)gf);
        while (g < A.n) {
            const float t = face_t(A, g);
            if (!(le ? t <= T : t < T)) break;
            ++g;
        }
        while (g > 0) {
            const float t = face_t(A, g - 1);
            if (le ? t <= T : t < T) break;
            --g;
        }
    }
    head = g < A.n ? face_t(A, g) : INFINITY;
    return g;
}

// Step j of axis Q: enters edge j + (the other axes' steps before it) + 1;
// returns that edge's index and sets its cell and range.
template <int Q>
__device__ __forceinline__ int walk_step(const WalkAxis (&ax)[3], int j, const RaySetup &r, int &c0, int &c1, int &c2,
                                         float &tin, float &tout) {
    constexpr int QA = Q == 0 ? 1 : 0, QB = Q == 2 ? 1 : 2;   // the other axes, QA < QB
    const WalkAxis &A = ax[Q], &Aa = ax[QA], &Ab = ax[QB];
    const float T = face_t(A, j);
    float ha, hb;
    const int ga = steps_before(Aa, T, QA < Q, ha);
    const int gb = steps_before(Ab, T, QB < Q, hb);
    const int i = j + ga + gb + 1;
    const int cq = A.s + A.dir * (j + 1), ca = Aa.s + Aa.dir * ga, cb = Ab.s + Ab.dir * gb;
    c0 = Q == 0 ? cq : ca;
    c1 = Q == 1 ? cq : (Q == 0 ? ca : cb);
    c2 = Q == 2 ? cq : cb;
    const float mi = T < r.t1 ? T : r.t1;
    tin = mi > r.t0 ? mi : r.t0;
    if (i == r.N - 1) {
        tout = r.t1;
    } else {
        float M = j + 1 < A.n ? face_t(A, j + 1) : INFINITY;
        M = ha < M ? ha : M;
        M = hb < M ? hb : M;
        const float mm = M < r.t1 ? M : r.t1;
        tout = mm > tin ? mm : tin;
    }
    return i;
}

constexpr int kWalkWarps = kThreads / 32;
constexpr int kWalkKeyTab = 1024;   // grids up to this many voxels per axis take the key tables
constexpr int kWalkQueue = 64;

__global__ void __launch_bounds__(kThreads, 3) k_ray_walk(const __grid_constant__ TravParams P,
                                                       const __grid_constant__ TravTables TT,
                                                       const RaySetup *__restrict__ setup,
                                                       const int64_t *__restrict__ ray_off, uint32_t *__restrict__ vox,
                                                       float *__restrict__ dmid, float *__restrict__ nu,
                                                       double *__restrict__ nu64, float *__restrict__ t_in,
                                                       float *__restrict__ t_out, float *__restrict__ wlen) {
    // the per-bin tables the edges index, copied to shared memory (indexed
    // loads from the kernel's parameter block are slow)
    __shared__ float s_inv[kMaxBins], s_thr[kMaxBins], s_ls[kMaxBins], s_bias[kMaxBins];
    __shared__ float q_d[kWalkWarps][kWalkQueue], q_Z[kWalkWarps][kWalkQueue];
    __shared__ int64_t q_e[kWalkWarps][kWalkQueue];
    // the voxel key is additive over the axes: (brick << 9) | Morton bits,
    // with the brick index linear in each axis's brick and the Morton bits of
    // different axes disjoint, so key = base + K_x[x] + K_y[y] + K_z[z]
    __shared__ uint32_t s_key[3][kWalkKeyTab];
    const bool key_tab = P.nx <= kWalkKeyTab && P.ny <= kWalkKeyTab && P.nz <= kWalkKeyTab;
    for (int i = threadIdx.x; i < P.n_bins; i += blockDim.x) {
        s_inv[i] = TT.far_inv_sig[i];
        s_thr[i] = TT.far_thr[i];
        s_ls[i] = TT.log_sigma[i];
        s_bias[i] = TT.bias[i];
    }
    if (key_tab) {
        const uint32_t stride[3] = {1u, P.nbx, P.nbx * P.nby};
        const int n[3] = {P.nx, P.ny, P.nz};
        for (int q = 0; q < 3; ++q)
            for (int c = threadIdx.x; c < n[q]; c += blockDim.x)
                s_key[q][c] = ((stride[q] * ((uint32_t)c >> 3)) << 9) | (spread3((uint32_t)c & 7u) << q);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    float *qd = q_d[wib], *qZ = q_Z[wib];
    int64_t *qe = q_e[wib];
    int qc = 0;   // queued FP64 evaluations (warp-uniform)
    const bool fp32_ctx = nu64 == nullptr;
    auto flush = [&](int cnt) {
        __syncwarp();
        if (lane < cnt) nu[qe[lane]] = (float)sensor_nu_f64(P, s_ls, s_bias, (double)qd[lane], (double)qZ[lane]);
        __syncwarp();
    };
    const int64_t npix = (int64_t)P.W * P.H;
    const int64_t nwarps = (int64_t)gridDim.x * kWalkWarps;
    for (int64_t p = (int64_t)blockIdx.x * kWalkWarps + wib; p < npix; p += nwarps) {
        const RaySetup r = setup[p];   // the same for every lane: broadcast loads
        if (r.N == 0) continue;
        const int64_t e0 = ray_off[p];
        WalkAxis ax[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ax[q].s = r.s[q];
            ax[q].n = r.e[q] > r.s[q] ? r.e[q] - r.s[q] : r.s[q] - r.e[q];
            ax[q].dir = r.k[q] > 0.0f ? 1 : -1;
            ax[q].base = r.s[q] + (r.k[q] > 0.0f ? 1 : 0);
            ax[q].o = P.o[q];
            ax[q].k = r.k[q];
            ax[q].inv = r.inv[q];
        }
        const int n01 = ax[0].n + ax[1].n;
        for (int m0 = 0; m0 < r.N; m0 += 32) {
            const int m = m0 + lane;
            const bool act = m < r.N;
            bool near = false;
            float d = 0.0f;
            int64_t e = 0;
            if (act) {
                int i, c0, c1, c2;
                float tin, tout;
                if (m == 0) {   // the first edge: the start cell, entered at t0
                    i = 0;
                    c0 = ax[0].s;
                    c1 = ax[1].s;
                    c2 = ax[2].s;
                    tin = r.t0;
                    float M = INFINITY;
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (ax[q].n > 0) {
                            const float t = face_t(ax[q], 0);
                            M = t < M ? t : M;
                        }
                    const float mm = M < r.t1 ? M : r.t1;
                    tout = r.N == 1 ? r.t1 : (mm > tin ? mm : tin);
                } else {        // step j of axis q, entering edge rank + 1
                    const int x = m - 1;
                    // the axis roles are compile-time constants in each case (the
                    // lanes of a warp mostly share q)
                    if (x < ax[0].n) i = walk_step<0>(ax, x, r, c0, c1, c2, tin, tout);
                    else if (x < n01) i = walk_step<1>(ax, x - ax[0].n, r, c0, c1, c2, tin, tout);
                    else i = walk_step<2>(ax, x - n01, r, c0, c1, c2, tin, tout);
                }
                const float sum = tin + tout;
                d = 0.5f * sum;
                e = e0 + i;
                vox[e] = P.key_base + (key_tab ? s_key[0][c0] + s_key[1][c1] + s_key[2][c2]
                                               : voxel_key((uint32_t)c0, (uint32_t)c1, (uint32_t)c2, P.nbx, P.nby));
                if (dmid) dmid[e] = d;
                if (t_in) t_in[e] = tin;
                if (t_out) t_out[e] = tout;
                if (wlen) wlen[e] = fminf(1.0f, (tout - tin) / P.h);   // traversed length in voxel edges, at most 1
                if (!fp32_ctx) {
                    const double v = sensor_nu_f64(P, s_ls, s_bias, (double)d, (double)r.Z);
                    nu64[e] = v;
                    if (nu) nu[e] = (float)v;
                } else if (nu) {
                    // edges far from the measured range skip the FP64
                    // evaluation, whose float would be the floor's anyway
                    if (P.far_ok && far_edge(P, s_inv, s_thr, d, r.Z)) nu[e] = P.w_floor;
                    else near = true;
                }
            }
            const uint32_t nm = __ballot_sync(0xffffffffu, near);
            if (nm) {
                if (near) {
                    const int pos = qc + __popc(nm & lt_mask);
                    qd[pos] = d;
                    qZ[pos] = r.Z;
                    qe[pos] = e;
                }
                qc += __popc(nm);
                if (qc >= 32) {
                    flush(32);
                    if (lane < qc - 32) {
                        qd[lane] = qd[32 + lane];
                        qZ[lane] = qZ[32 + lane];
                        qe[lane] = qe[32 + lane];
                    }
                    qc -= 32;
                }
            }
        }
    }
    if (qc > 0) flush(qc);
}

// a warp per ray over a grid the SMs hold at once (each warp takes every
// nwarps-th ray), so that a warp's FP64 queue fills across several rays
unsigned walk_blocks(int64_t npix) {
    static int cap = 0;
    if (cap == 0) {
        int dev = 0, nsm = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ray_walk, kThreads, 0) != cudaSuccess)
            nsm = per_sm = 1;
        cap = nsm * (per_sm > 0 ? per_sm : 1);
    }
    const int64_t need = ceil_div(npix, (int64_t)kWalkWarps);
    return (unsigned)(need < cap ? need : cap);
}

}  // namespace

cudaError_t launch_ray_setup(const TravParams &P, const TravTables &TT, const float *depth, int32_t *counts,
                             float *Zr, int32_t *max_len, void *setup, cudaStream_t s) {
    const int64_t npix = (int64_t)P.W * P.H;
    if (npix == 0) return cudaSuccess;
    k_ray_setup<<<(unsigned)ceil_div(npix, kThreads), kThreads, 0, s>>>(P, TT, depth, counts, Zr, max_len,
                                                                        static_cast<RaySetup *>(setup));
    return cudaGetLastError();
}

cudaError_t launch_ray_walk(const TravParams &P, const TravTables &TT, const void *setup, const int64_t *ray_off,
                            uint32_t *vox, float *dmid, float *nu, double *nu64, float *wlen, cudaStream_t s) {
    const int64_t npix = (int64_t)P.W * P.H;
    if (npix == 0) return cudaSuccess;
    k_ray_walk<<<walk_blocks(npix), kThreads, 0, s>>>(P, TT, static_cast<const RaySetup *>(setup), ray_off, vox, dmid, nu,
                                                      nu64, nullptr, nullptr,
                                                      wlen);
    return cudaGetLastError();
}

cudaError_t launch_ray_walk_seg(const TravParams &P, const TravTables &TT, const void *setup, const int64_t *ray_off,
                                uint32_t *vox, float *t_in, float *t_out, cudaStream_t s) {
    const int64_t npix = (int64_t)P.W * P.H;
    if (npix == 0) return cudaSuccess;
    k_ray_walk<<<walk_blocks(npix), kThreads, 0, s>>>(P, TT, static_cast<const RaySetup *>(setup), ray_off, vox, nullptr,
                                                      nullptr, nullptr, t_in,
                                                      t_out, nullptr);
    return cudaGetLastError();
}

}  // namespace mrf
