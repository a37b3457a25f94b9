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

struct RaySetup {
    float k[3], inv[3];
    float t0, t1, Z;
    int s[3], e[3];
    int N;
};

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
                                                        float *__restrict__ Zr, int32_t *__restrict__ max_len) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = (int64_t)P.W * P.H;
    int N = 0;
    if (p < npix) {
        RaySetup r;
        ray_setup(P, TT, (int)(p % P.W), (int)(p / P.W), depth[p], r);
        N = r.N;
        counts[p] = N;
        Zr[p] = r.Z;
    }
    // warp max, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) N = max(N, __shfl_xor_sync(0xffffffffu, N, o));
    if ((threadIdx.x & 31) == 0 && N > 0) atomicMax(max_len, N);
}

__global__ void __launch_bounds__(kThreads) k_ray_walk(const __grid_constant__ TravParams P,
                                                       const __grid_constant__ TravTables TT,
                                                       const float *__restrict__ depth,
                                                       const int64_t *__restrict__ ray_off, uint32_t *__restrict__ vox,
                                                       float *__restrict__ dmid, float *__restrict__ nu,
                                                       double *__restrict__ nu64, float *__restrict__ t_in,
                                                       float *__restrict__ t_out, float *__restrict__ wlen) {
    // the per-bin tables the edges index, copied to shared memory (indexed
    // loads from the kernel's parameter block are slow)
    __shared__ float s_inv[kMaxBins], s_thr[kMaxBins], s_ls[kMaxBins], s_bias[kMaxBins];
    for (int i = threadIdx.x; i < P.n_bins; i += blockDim.x) {
        s_inv[i] = TT.far_inv_sig[i];
        s_thr[i] = TT.far_thr[i];
        s_ls[i] = TT.log_sigma[i];
        s_bias[i] = TT.bias[i];
    }
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = (int64_t)P.W * P.H;
    if (p >= npix) return;
    RaySetup r;
    ray_setup(P, TT, (int)(p % P.W), (int)(p / P.W), depth[p], r);
    if (r.N == 0) return;
    const int64_t e0 = ray_off[p];
    int c[3] = {r.s[0], r.s[1], r.s[2]};
    float tin = r.t0;
    // edge i of the ray: its key, midpoint range and likelihood (the optional
    // per-edge outputs stored here); advances the walk
    auto edge = [&](int i, uint32_t &key, float &dm, float &lik) {
        float tout;
        int best = -1;
        if (i == r.N - 1) {
            tout = r.t1;
        } else {
            float bt = 0.0f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (c[q] == r.e[q]) continue;
                const float bound = (float)(c[q] + (r.k[q] > 0.0f ? 1 : 0));
                const float tm = (bound - P.o[q]) * r.inv[q];
                if (best < 0 || tm < bt) {
                    best = q;
                    bt = tm;
                }
            }
            const float m = bt < r.t1 ? bt : r.t1;
            tout = m > tin ? m : tin;
        }
        const float s = tin + tout;
        const float d = 0.5f * s;
        const int64_t e = e0 + i;
        key = P.key_base + voxel_key((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2], P.nbx, P.nby);
        dm = d;
        lik = 0.0f;
        if (t_in) t_in[e] = tin;
        if (t_out) t_out[e] = tout;
        if (wlen) wlen[e] = fminf(1.0f, (tout - tin) / P.h);   // traversed length in voxel edges, at most 1
        if (nu || nu64) {
            // FP32 contexts: edges far from the measured range skip the FP64
            // evaluation, whose float would be the floor's anyway
            if (!nu64 && P.far_ok && far_edge(P, s_inv, s_thr, d, r.Z)) {
                lik = P.w_floor;
            } else {
                const double v = sensor_nu_f64(P, s_ls, s_bias, (double)d, (double)r.Z);
                lik = (float)v;
                if (nu64) nu64[e] = v;
            }
        }
        if (best >= 0) {
            // (a constant index per axis keeps c and r in registers)
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q == best) c[q] += r.k[q] > 0.0f ? 1 : -1;
            tin = tout;
        }
    };
    // Each thread writes its own ray's run of the edge arrays; 16-byte stores
    // of four edges (after a head that reaches a multiple of four) fill a
    // sector's half where single stores filled an eighth.
    int i = 0;
    for (; i < r.N && ((e0 + i) & 3); ++i) {
        uint32_t key;
        float dm, lik;
        edge(i, key, dm, lik);
        vox[e0 + i] = key;
        if (dmid) dmid[e0 + i] = dm;
        if (nu) nu[e0 + i] = lik;
    }
    for (; i + 4 <= r.N; i += 4) {
        uint32_t key[4];
        float dm[4], lik[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) edge(i + u, key[u], dm[u], lik[u]);
        const int64_t e = e0 + i;
        *reinterpret_cast<uint4 *>(vox + e) = make_uint4(key[0], key[1], key[2], key[3]);
        if (dmid) *reinterpret_cast<float4 *>(dmid + e) = make_float4(dm[0], dm[1], dm[2], dm[3]);
        if (nu) *reinterpret_cast<float4 *>(nu + e) = make_float4(lik[0], lik[1], lik[2], lik[3]);
    }
    for (; i < r.N; ++i) {
        uint32_t key;
        float dm, lik;
        edge(i, key, dm, lik);
        vox[e0 + i] = key;
        if (dmid) dmid[e0 + i] = dm;
        if (nu) nu[e0 + i] = lik;
    }
}

}  // namespace

cudaError_t launch_ray_setup(const TravParams &P, const TravTables &TT, const float *depth, int32_t *counts,
                             float *Zr, int32_t *max_len, cudaStream_t s) {
    const int64_t npix = (int64_t)P.W * P.H;
    if (npix == 0) return cudaSuccess;
    k_ray_setup<<<(unsigned)ceil_div(npix, kThreads), kThreads, 0, s>>>(P, TT, depth, counts, Zr, max_len);
    return cudaGetLastError();
}

cudaError_t launch_ray_walk(const TravParams &P, const TravTables &TT, const float *depth, const int64_t *ray_off,
                            uint32_t *vox, float *dmid, float *nu, double *nu64, float *wlen, cudaStream_t s) {
    const int64_t npix = (int64_t)P.W * P.H;
    if (npix == 0) return cudaSuccess;
    k_ray_walk<<<(unsigned)ceil_div(npix, kThreads), kThreads, 0, s>>>(P, TT, depth, ray_off, vox, dmid, nu, nu64,
                                                                       nullptr, nullptr, wlen);
    return cudaGetLastError();
}

cudaError_t launch_ray_walk_seg(const TravParams &P, const TravTables &TT, const float *depth, const int64_t *ray_off,
                                uint32_t *vox, float *t_in, float *t_out, cudaStream_t s) {
    const int64_t npix = (int64_t)P.W * P.H;
    if (npix == 0) return cudaSuccess;
    k_ray_walk<<<(unsigned)ceil_div(npix, kThreads), kThreads, 0, s>>>(P, TT, depth, ray_off, vox, nullptr, nullptr,
                                                                       nullptr, t_in, t_out, nullptr);
    return cudaGetLastError();
}

}  // namespace mrf
