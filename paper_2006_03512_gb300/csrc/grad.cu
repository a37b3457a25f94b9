// Gradient of a held-out depth likelihood with respect to the noise table.
//
// Not in the paper (it fits the table offline, Section IV-C).  The map's edges
// (voxels, midpoint ranges d, each ray's measured range Z) stay fixed; the
// table theta = (log sigma at the bin centres, outlier weight w) enters every
// edge's likelihood nu and nu_bg = w / d_hi.  The loss is
//   -sum_r log S_r,  S_r = sum_i nu_i p_{v_i} Q_i + nu_bg Q_{N+1},
//   Q_i = prod_{k<i} (1 - p_{v_k}),
// over held-out rays, with p the marginals after the unrolled BP passes: the
// probability of the measured depth when each voxel's occupancy is drawn from
// its marginal (Eq. "depth_message" summed over the first occupied voxel).
//
// The reverse pass runs one warp per ray in FP32 (the forward kernel's
// excess form), over the FP32 forward's per-pass checkpoints (messages and
// voxel totals); per-edge adjoints are kept in FP64, per-voxel sums go through
// the deterministic segmented reduction and the table gradient through fixed-
// order block sums, so the result is bitwise reproducible.  Edges far from
// their ray's measured range (ThetaTab's far distances, set on the host) skip
// the FP64 exponentials: their likelihood is the floor's float and their
// table partials are 0 and 1 / d_hi, to 2^-40 relative.
#include <cmath>

#include "mrf_internal.cuh"

namespace mrf {
namespace {

// table position of range d: bin k and weight f of bin k+1 (the rule of the
// likelihood in traverse.cu)
__device__ __forceinline__ void theta_pos(const ThetaTab &th, double d, int &k, double &f) {
    const double x = (d - th.dlo) / th.delta - 0.5;
    const double fk = floor(x);
    if (!(fk >= 0.0)) k = 0;
    else if (fk > th.n_bins - 2) k = th.n_bins - 2;
    else k = (int)fk;
    f = x - k;
    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
}

// nu(d | Z; theta) = (1 - w) N(Z; d + b(d), sigma(d)) + w / d_hi, and its
// partials with respect to log sigma(d) and w
__device__ __forceinline__ double theta_nu(const ThetaTab &th, double d, double Z, int &k, double &f, double &dls,
                                           double &dw) {
    theta_pos(th, d, k, f);
    const double ls = (1.0 - f) * th.ls[k] + f * th.ls[k + 1];
    const double b = th.has_bias ? (1.0 - f) * (double)th.bias[k] + f * (double)th.bias[k + 1] : 0.0;
    const double zz = (Z - (d + b)) * exp(-ls);
    const double G = exp(-0.5 * zz * zz - ls - 0.91893853320467274178);
    dls = (1.0 - th.w) * G * (zz * zz - 1.0);
    dw = -G + 1.0 / th.dhi;
    if (th.w <= 0.0) return G;
    return (1.0 - th.w) * G + th.w / th.dhi;
}

// |Z - d| beyond the far distance of the edge's FP32 table bin (see ThetaTab):
// there the Gaussian part is below 2^-40 of the floor.  The FP32 bin can be
// off by one from the exact one; far_d[k] covers bins k - 1 .. k + 1.
__device__ __forceinline__ bool theta_far(const ThetaTab &th, float d, float Z) {
    const float x = floorf(fmaf(d - th.dlo_f, th.inv_delta_f, -0.5f));
    const int k = (int)fminf(fmaxf(x, 0.f), (float)(th.n_bins - 2));
    return fabsf(Z - d) > th.far_d[k];
}

// The likelihood of every edge under theta, a warp per ray (lanes over its
// edges); far edges take the floor's float without the exponentials.
__global__ void k_nu_theta(const __grid_constant__ ThetaTab th, const int64_t *__restrict__ ray_off, int64_t R,
                           const float *__restrict__ dmid, const float *__restrict__ Zr, float *__restrict__ nu) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= R) return;
    const float Z = Zr[r];
    const int64_t e1 = ray_off[r + 1];
    for (int64_t e = ray_off[r] + (threadIdx.x & 31); e < e1; e += 32) {
        const float d = dmid[e];
        if (th.far_ok && theta_far(th, d, Z)) {
            nu[e] = th.nu_far;
        } else {
            int k;
            double f, dls, dw;
            nu[e] = (float)theta_nu(th, (double)d, (double)Z, k, f, dls, dw);
        }
    }
}

__device__ __forceinline__ double sigmoid_d(double t) { return 1.0 / (1.0 + exp(-t)); }

// Held-out rays, one thread each: loss_r, and d loss / d p at each edge (gp),
// d loss / d nu (gnu), d loss / d nu_bg (gbg per ray).  Q holds the prefix
// products (the backward sweep cannot divide by 1 - p when p = 1).
__global__ void k_heldout(const __grid_constant__ ThetaTab th, const int64_t *__restrict__ ray_off, int64_t R,
                          const uint32_t *__restrict__ vox, const float *__restrict__ dmid,
                          const float *__restrict__ Zr, const float *__restrict__ T, double nu_bg,
                          double *__restrict__ Q, double *__restrict__ nuh, double *__restrict__ gp,
                          double *__restrict__ gnu, double *__restrict__ loss_r, double *__restrict__ gbg) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t e0 = ray_off[r], e1 = ray_off[r + 1];
    if (e1 == e0) {
        loss_r[r] = 0.0;
        gbg[r] = 0.0;
        return;
    }
    const float Zf = Zr[r];
    const double Z = Zf, floor_d = th.w > 0.0 ? th.w / th.dhi : 0.0;
    double S = 0.0, q = 1.0;
    for (int64_t e = e0; e < e1; ++e) {
        const float d = dmid[e];
        double n;
        if (theta_far(th, d, Zf)) {   // the floor, to 2^-40 relative
            n = floor_d;
        } else {
            int k;
            double f, dls, dw;
            n = theta_nu(th, (double)d, Z, k, f, dls, dw);
        }
        const double pv = sigmoid_d((double)T[vox[e]]);
        nuh[e] = n;
        Q[e] = q;
        gp[e] = pv;   // kept for the backward sweep, which overwrites it
        S += n * pv * q;
        q *= 1.0 - pv;
    }
    S += nu_bg * q;
    loss_r[r] = -log(S);
    const double gS = -1.0 / S;
    gbg[r] = gS * q;
    double Rs = nu_bg;   // sum_{j>i} nu_j p_j prod_{i<k<j}(1 - p_k) + nu_bg prod_{k>i}(1 - p_k)
    for (int64_t e = e1 - 1; e >= e0; --e) {
        const double pv = gp[e];
        gp[e] = gS * Q[e] * (nuh[e] - Rs);
        gnu[e] = gS * pv * Q[e];
        Rs = nuh[e] * pv + (1.0 - pv) * Rs;
    }
}

// d loss / d T = d loss / d p * p (1 - p), over every voxel key
__global__ void k_sigmoid_adjoint(const float *__restrict__ T, double *__restrict__ g, int64_t V) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const double p = sigmoid_d((double)T[v]);
    g[v] *= p * (1.0 - p);
}

// d loss / d lambda^(t)_e = d loss / d T^(t)[v_e] - d loss / d L^(t+1)_e
// (T^(t) = logit gamma + sum lambda^(t); L^(t+1) = T^(t)[v] - lambda^(t))
__global__ void k_glam(const double *__restrict__ gT, const uint32_t *__restrict__ vox,
                       const double *__restrict__ gLn, int64_t E, double *__restrict__ glam) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E) glam[e] = gT[vox[e]] - gLn[e];
}

// Reverse mode of the ray messages (Eqs. "pos"/"neg"), one warp per ray, in
// FP32 on the forward kernel's excess form (ray_tile.cuh): with c the
// likelihood floor, nu' = nu - c, P_{i+1} = P_i m0_i, A'_{i+1} = A'_i +
// P_i m1_i nu'_i, beta_{i-1} = m1_i nu'_i + m0_i beta_i (beta after the last
// voxel: nu_bg - c), lambda_i = log(num_i / den_i), num_i = c + A'_i + P_i
// nu'_i, den_i = c + A'_i + P_i beta_i.  The partials of lambda_i are formed
// without cancellation:
//   d/dA'   = 1/num - 1/den = -P (nu' - beta) / (num den)
//   d/dP    = nu'/num - beta/den = (nu' - beta)(c + A') / (num den)
//   d/dnu'  = P / num,  d/dbeta = -P / den.
// Three sweeps: forward (P, A'), backward (beta and the adjoints of A' and P),
// forward (the adjoint of beta).  Cavities are the FP32 ones the forward used:
// L0 in the first pass, else T^(t-1)[v] - lambda^(t-1), gathered once (first
// sweep) and kept.  Writes gL, adds into gnu and gbg (per ray).  A message the
// forward clamps to +-64 passes no gradient.  Scratch (FP32 per edge): the
// cavity; P; A' then d/dm; beta; d/dbeta.
__device__ __forceinline__ void sigmoid_pair(float L, float &m1, float &m0) {
    const float e = __expf(-fabsf(L));
    const float r = 1.f / (1.f + e);
    const float sm = e * r;
    m1 = L < 0.f ? sm : r;
    m0 = L < 0.f ? r : sm;
}

// Each lane holds kAdjK consecutive edges of a 32 * kAdjK-edge chunk, every
// sweep is a warp scan of affine maps per chunk (chunks in order, the state
// carried between them), and every load and store is coalesced.  The sweeps:
//   forward   (A', P) <- (A' + P m1 nu', P m0)                 [stores P, A', L]
//   backward  beta <- m1 nu' + m0 beta, then the message partials, then
//             (Abar, Pbar) <- (Abar + dA, m1 nu' Abar + m0 Pbar + dP)
//                                                              [stores beta, d/dbeta, d/dm]
//   forward   Bbar <- d/dbeta + m0 Bbar                        [writes gL, adds gnu]
constexpr int kAdjK = 4;

struct Aff1 {   // x -> u + v x
    float u, v;
};
struct Aff2 {   // (a, p) -> (a + A, q a + r p + B)
    float q, r, A, B;
};
__device__ __forceinline__ Aff1 aff1_then(const Aff1 &f, const Aff1 &g) {   // f first, then g
    return {fmaf(g.v, f.u, g.u), g.v * f.v};
}
__device__ __forceinline__ Aff2 aff2_then(const Aff2 &f, const Aff2 &g) {   // f first, then g
    return {fmaf(g.r, f.q, g.q), g.r * f.r, f.A + g.A, fmaf(g.q, f.A, fmaf(g.r, f.B, g.B))};
}
__device__ __forceinline__ Aff1 shfl1(const Aff1 &a, int src_delta, bool up) {
    return up ? Aff1{__shfl_up_sync(0xffffffffu, a.u, src_delta), __shfl_up_sync(0xffffffffu, a.v, src_delta)}
              : Aff1{__shfl_down_sync(0xffffffffu, a.u, src_delta), __shfl_down_sync(0xffffffffu, a.v, src_delta)};
}
__device__ __forceinline__ Aff2 shfl2_down(const Aff2 &a, int d) {
    return {__shfl_down_sync(0xffffffffu, a.q, d), __shfl_down_sync(0xffffffffu, a.r, d),
            __shfl_down_sync(0xffffffffu, a.A, d), __shfl_down_sync(0xffffffffu, a.B, d)};
}
// the forward state map (A, P) -> (A + u P, v P), stored in an Aff1: f first, then g
__device__ __forceinline__ Aff1 ap_then(const Aff1 &f, const Aff1 &g) { return {fmaf(f.v, g.u, f.u), f.v * g.v}; }
// exclusive scan of lane maps in lane order (lane 0 first): the composition of
// the maps of lanes < lane, and the warp total (AP: the (A, P) composition,
// else x -> u + v x)
template <bool AP>
__device__ __forceinline__ Aff1 warp_excl_fwd(Aff1 m, Aff1 &total) {
    const int lane = threadIdx.x & 31;
    Aff1 inc = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Aff1 y = shfl1(inc, o, true);
        if (lane >= o) inc = AP ? ap_then(y, inc) : aff1_then(y, inc);
    }
    total = {__shfl_sync(0xffffffffu, inc.u, 31), __shfl_sync(0xffffffffu, inc.v, 31)};
    Aff1 ex = shfl1(inc, 1, true);
    if (lane == 0) ex = {0.f, 1.f};
    return ex;
}
// exclusive scan in reverse lane order (lane 31 first)
__device__ __forceinline__ Aff1 warp_excl_bwd(Aff1 m, Aff1 &total) {
    const int lane = threadIdx.x & 31;
    Aff1 inc = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Aff1 y = shfl1(inc, o, false);
        if (lane + o < 32) inc = aff1_then(y, inc);
    }
    total = {__shfl_sync(0xffffffffu, inc.u, 0), __shfl_sync(0xffffffffu, inc.v, 0)};
    Aff1 ex = shfl1(inc, 1, false);
    if (lane == 31) ex = {0.f, 1.f};
    return ex;
}
__device__ __forceinline__ Aff2 warp_excl_bwd2(Aff2 m, Aff2 &total) {
    const int lane = threadIdx.x & 31;
    Aff2 inc = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Aff2 y = shfl2_down(inc, o);
        if (lane + o < 32) inc = aff2_then(y, inc);
    }
    total = {__shfl_sync(0xffffffffu, inc.q, 0), __shfl_sync(0xffffffffu, inc.r, 0),
             __shfl_sync(0xffffffffu, inc.A, 0), __shfl_sync(0xffffffffu, inc.B, 0)};
    Aff2 ex = shfl2_down(inc, 1);
    if (lane == 31) ex = {0.f, 1.f, 0.f, 0.f};
    return ex;
}

__global__ void __launch_bounds__(128) k_ray_adjoint_warp(
    const int64_t *__restrict__ ray_off, int64_t R, const uint32_t *__restrict__ vox, const float *__restrict__ nu,
    const float *__restrict__ Tprev, const float *__restrict__ lprev, float L0, int first, float nu_bg, float c,
    const double *__restrict__ glam, float *__restrict__ sL, float *__restrict__ sP, float *__restrict__ sA,
    float *__restrict__ sB, float *__restrict__ sD, double *__restrict__ gL, double *__restrict__ gnu,
    double *__restrict__ gbg) {
    constexpr int C = 32 * kAdjK;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= R) return;   // the whole warp leaves together
    const int lane = threadIdx.x & 31;
    const int64_t e0 = ray_off[r], e1 = ray_off[r + 1];
    const int64_t N = e1 - e0;
    if (N == 0) return;
    const int nch = (int)((N + C - 1) / C);
    // forward: (A', P) as the map (A, P) -> (A + x P, y P): Aff1 with u = x, v = y
    float cA = 0.f, cP = 1.f;   // state entering the chunk
    for (int ch = 0; ch < nch; ++ch) {
        const int64_t b0 = e0 + (int64_t)ch * C + lane * kAdjK;
        float L[kAdjK], m1[kAdjK], m0[kAdjK], cc[kAdjK];
        Aff1 agg = {0.f, 1.f};
#pragma unroll
        for (int k = 0; k < kAdjK; ++k) {
            const int64_t e = b0 + k;
            L[k] = 0.f;
            m1[k] = 0.f;
            m0[k] = 1.f;
            cc[k] = 0.f;
            if (e < e1) {
                L[k] = first ? L0 : Tprev[vox[e]] - lprev[e];
                sigmoid_pair(L[k], m1[k], m0[k]);
                cc[k] = m1[k] * (nu[e] - c);
                agg = {fmaf(agg.v, cc[k], agg.u), agg.v * m0[k]};
            }
        }
        Aff1 tot;
        const Aff1 ex = warp_excl_fwd<true>(agg, tot);
        float A = fmaf(cP, ex.u, cA), P = cP * ex.v;
#pragma unroll
        for (int k = 0; k < kAdjK; ++k) {
            const int64_t e = b0 + k;
            if (e < e1) {
                sL[e] = L[k];
                sP[e] = P;
                sA[e] = A;
                A = fmaf(P, cc[k], A);
                P *= m0[k];
            }
        }
        cA = fmaf(cP, tot.u, cA);
        cP *= tot.v;
    }
    // backward over the chunks, last first
    float cB = nu_bg - c;                  // beta after the chunk's last edge
    float cAb = 0.f, cPb = 0.f;            // (Abar, Pbar) after it
    for (int ch = nch - 1; ch >= 0; --ch) {
        const int64_t b0 = e0 + (int64_t)ch * C + lane * kAdjK;
        float m1[kAdjK], m0[kAdjK], nx[kAdjK], Pi[kAdjK], Ai[kAdjK];
        bool in[kAdjK];
        // beta: the map beta_i -> beta_{i-1} = m1 nu' + m0 beta_i, composed from the
        // lane's last edge to its first
        Aff1 bagg = {0.f, 1.f};
#pragma unroll
        for (int k = kAdjK - 1; k >= 0; --k) {
            const int64_t e = b0 + k;
            in[k] = e < e1;
            m1[k] = 0.f;
            m0[k] = 1.f;
            nx[k] = 0.f;
            Pi[k] = 0.f;
            Ai[k] = 0.f;
            if (in[k]) {
                sigmoid_pair(sL[e], m1[k], m0[k]);
                nx[k] = nu[e] - c;
                Pi[k] = sP[e];
                Ai[k] = sA[e];
                bagg = aff1_then(bagg, Aff1{m1[k] * nx[k], m0[k]});
            }
        }
        Aff1 btot;
        const Aff1 bex = warp_excl_bwd(bagg, btot);
        // beta at each edge (the state after it, from the right)
        float Bv[kAdjK], dA[kAdjK], dP[kAdjK], dnu[kAdjK], dB[kAdjK];
        {
            float B = fmaf(bex.v, cB, bex.u);
#pragma unroll
            for (int k = kAdjK - 1; k >= 0; --k) {
                Bv[k] = B;
                if (in[k]) B = fmaf(m1[k], nx[k], m0[k] * B);
            }
        }
        // message partials, then the lane's (Abar, Pbar) map from its last edge to its first
        Aff2 agg2 = {0.f, 1.f, 0.f, 0.f};
#pragma unroll
        for (int k = kAdjK - 1; k >= 0; --k) {
            dA[k] = dP[k] = dnu[k] = dB[k] = 0.f;
            if (in[k]) {
                const int64_t e = b0 + k;
                const float base = c + Ai[k];
                const float num = fmaf(Pi[k], nx[k], base), den = fmaf(Pi[k], Bv[k], base);
                const float lam = __logf(num) - __logf(den);
                const bool live = lam == lam && fabsf(lam) < kLamClamp - 1e-3f;
                const float g = (float)glam[e];
                const float gn = live ? g / num : 0.f, gd = live ? gn / den : 0.f, gdn = live ? g / den : 0.f;
                dA[k] = -gd * Pi[k] * (nx[k] - Bv[k]);
                dP[k] = gd * (nx[k] - Bv[k]) * base;
                dnu[k] = gn * Pi[k];
                dB[k] = -gdn * Pi[k];
                // (Abar, Pbar)_i = (Abar_{i+1} + dA, m1 nu' Abar_{i+1} + m0 Pbar_{i+1} + dP)
                agg2 = aff2_then(agg2, Aff2{m1[k] * nx[k], m0[k], dA[k], dP[k]});
            }
        }
        Aff2 tot2;
        const Aff2 ex2 = warp_excl_bwd2(agg2, tot2);
        float Ab = cAb + ex2.A, Pb = fmaf(ex2.q, cAb, fmaf(ex2.r, cPb, ex2.B));
#pragma unroll
        for (int k = kAdjK - 1; k >= 0; --k) {
            if (in[k]) {
                const int64_t e = b0 + k;
                const float gm = (Ab * nx[k] - Pb) * Pi[k];   // d/dm1 from A'_{i+1}, minus d/dm0 from P_{i+1}
                gnu[e] += (double)fmaf(Ab * Pi[k], m1[k], dnu[k]);
                sA[e] = gm;
                sB[e] = Bv[k];
                sD[e] = dB[k];
                const float Pn = dP[k] + Ab * m1[k] * nx[k] + Pb * m0[k];
                Ab += dA[k];
                Pb = Pn;
            }
        }
        cB = fmaf(btot.v, cB, btot.u);
        const float nAb = cAb + tot2.A;
        cPb = fmaf(tot2.q, cAb, fmaf(tot2.r, cPb, tot2.B));
        cAb = nAb;
    }
    // forward: Bbar_i = d/dbeta_i + m0_i Bbar_{i-1}
    float cBb = 0.f;
    bool started = false;
    for (int ch = 0; ch < nch; ++ch) {
        const int64_t b0 = e0 + (int64_t)ch * C + lane * kAdjK;
        float m1[kAdjK], m0[kAdjK];
        Aff1 agg = {0.f, 1.f};
#pragma unroll
        for (int k = 0; k < kAdjK; ++k) {
            const int64_t e = b0 + k;
            m1[k] = 0.f;
            m0[k] = 1.f;
            if (e < e1) {
                sigmoid_pair(sL[e], m1[k], m0[k]);
                agg = aff1_then(agg, Aff1{sD[e], m0[k]});
            }
        }
        Aff1 tot;
        const Aff1 ex = warp_excl_fwd<false>(agg, tot);
        float Bb = fmaf(ex.v, cBb, ex.u);   // Bbar_{i-1} entering the lane's first edge
#pragma unroll
        for (int k = 0; k < kAdjK; ++k) {
            const int64_t e = b0 + k;
            if (e < e1) {
                float gm = sA[e];
                if (e > e0) {
                    gm = fmaf(Bb, (nu[e] - c) - sB[e], gm);   // d/dm1 gets Bbar nu', d/dm0 gets Bbar beta
                    gnu[e] += (double)(Bb * m1[k]);
                }
                Bb = fmaf(m0[k], Bb, sD[e]);
                gL[e] = (double)(gm * m1[k] * m0[k]);
            }
        }
        cBb = fmaf(tot.v, cBb, tot.u);
        started = true;
    }
    if (lane == 0 && started) gbg[r] += (double)cBb;
}

// Table gradient: sum over edges of g_nu * d nu / d theta.  A warp walks its
// rays, its lanes over each ray's edges, and each lane adds into its own
// shared-memory row; far edges only add g_nu / d_hi to the w entry (summed in
// a register first).  Rows are then summed in thread order, giving one partial
// per block (n_bins + 1 doubles; w last).
__global__ void k_theta_grad(const __grid_constant__ ThetaTab th, const int64_t *__restrict__ ray_off, int64_t R,
                             const float *__restrict__ dmid, const float *__restrict__ Zr,
                             const double *__restrict__ gnu, double *__restrict__ part) {
    extern __shared__ double rows[];   // blockDim.x rows of n_bins + 1
    const int nb = th.n_bins + 1;
    double *mine = rows + (size_t)threadIdx.x * nb;
    for (int k = 0; k < nb; ++k) mine[k] = 0.0;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double gfar = 0.0;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R; r += nw) {
        const float Z = Zr[r];
        const int64_t e1 = ray_off[r + 1];
        for (int64_t e = ray_off[r] + (threadIdx.x & 31); e < e1; e += 32) {
            const float d = dmid[e];
            const double g = gnu[e];
            if (theta_far(th, d, Z)) {
                gfar += g;
                continue;
            }
            int k;
            double f, dls, dw;
            theta_nu(th, (double)d, (double)Z, k, f, dls, dw);
            mine[k] += g * dls * (1.0 - f);
            mine[k + 1] += g * dls * f;
            mine[nb - 1] += g * dw;
        }
    }
    mine[nb - 1] += gfar / th.dhi;
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) s += rows[(size_t)t * nb + k];
        part[(size_t)blockIdx.x * nb + k] = s;
    }
}

// The accuracy metric of Section "Evaluation Metric for Probabilistic
// Occupancy Maps", one thread per ray walked to the grid exit.  Readings:
// alpha_i = -log(1 - p_i) / h (a ray crossing a whole voxel keeps visibility
// 1 - p_i); omega = alpha vis is largest, inside a voxel, at its entry, so the
// most likely generating surface is the voxel with the largest alpha_i vis_i
// (first on ties); the visibility left at the boundary is the chance the
// surface lies beyond the map, chosen when it exceeds that voxel's occlusion
// mass vis_i - vis_{i+1}.  A ray is accurate when its range Z falls in the
// chosen voxel's [entry, exit), or beyond the boundary when Z passes the
// exit of its last voxel.  p is the marginal as mrf_marginals writes it.
template <class V>
__global__ void k_omega(const int64_t *__restrict__ ray_off, int64_t R, const uint32_t *__restrict__ vox,
                        const float *__restrict__ t_in, const float *__restrict__ t_out, const float *__restrict__ Zr,
                        const V *__restrict__ T, double h, int8_t *__restrict__ result,
                        unsigned long long *__restrict__ counts) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t e0 = ray_off[r], e1 = ray_off[r + 1];
    if (e1 == e0) {
        if (result) result[r] = -1;
        return;
    }
    double vis = 1.0, best_w = -1.0, best_mass = 0.0;
    int64_t best = -1;
    for (int64_t e = e0; e < e1; ++e) {
        const V t = T[vox[e]];
        const double p = (double)(float)((V)1 / ((V)1 + exp(-t)));   // the marginal as mrf_marginals rounds it
        const double l = (double)t_out[e] - (double)t_in[e];
        const double a = p >= 1.0 ? (double)INFINITY : -log1p(-p) / h;
        const double w = a * vis;   // an occupied voxel behind a fully occluded one gives NaN: never a maximum
        const double vn = p >= 1.0 ? (l > 0.0 ? 0.0 : vis) : vis * exp(-a * l);
        if (w > best_w) {
            best_w = w;
            best = e;
            best_mass = vis - vn;
        }
        vis = vn;
    }
    const float Z = Zr[r];
    int acc;
    if (best < 0 || vis > best_mass) acc = Z > t_out[e1 - 1];
    else acc = t_in[best] <= Z && Z < t_out[best];
    if (result) result[r] = (int8_t)acc;
    atomicAdd(&counts[0], (unsigned long long)acc);
    atomicAdd(&counts[1], 1ull);
}

inline unsigned nblk(int64_t n, int t = kThreads) { return (unsigned)ceil_div(n > 0 ? n : 1, t); }

}  // namespace

cudaError_t launch_nu_theta(const ThetaTab &th, const int64_t *ray_off, int64_t R, const float *dmid,
                            const float *Zr, float *nu, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    k_nu_theta<<<nblk(R * 32, 128), 128, 0, s>>>(th, ray_off, R, dmid, Zr, nu);
    return cudaGetLastError();
}

cudaError_t launch_heldout(const ThetaTab &th, const int64_t *ray_off, int64_t R, const uint32_t *vox,
                           const float *dmid, const float *Zr, const float *T, double nu_bg, double *Q, double *nuh,
                           double *gp, double *gnu, double *loss_r, double *gbg, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    k_heldout<<<nblk(R, 128), 128, 0, s>>>(th, ray_off, R, vox, dmid, Zr, T, nu_bg, Q, nuh, gp, gnu, loss_r, gbg);
    return cudaGetLastError();
}

cudaError_t launch_sigmoid_adjoint(const float *T, double *g, int64_t V, cudaStream_t s) {
    k_sigmoid_adjoint<<<nblk(V), kThreads, 0, s>>>(T, g, V);
    return cudaGetLastError();
}

cudaError_t launch_glam(const double *gT, const uint32_t *vox, const double *gLn, int64_t E, double *glam,
                        cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    k_glam<<<nblk(E), kThreads, 0, s>>>(gT, vox, gLn, E, glam);
    return cudaGetLastError();
}

cudaError_t launch_ray_adjoint(const int64_t *ray_off, int64_t R, const uint32_t *vox, const float *nu,
                               const float *Tprev, const float *lprev, float L0, int first, float nu_bg,
                               float nu_ref, const double *glam, float *sL, float *sP, float *sA, float *sB,
                               float *sD, double *gL, double *gnu, double *gbg, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    k_ray_adjoint_warp<<<nblk(R * 32, 128), 128, 0, s>>>(ray_off, R, vox, nu, Tprev, lprev, L0, first, nu_bg, nu_ref,
                                                         glam, sL, sP, sA, sB, sD, gL, gnu, gbg);
    return cudaGetLastError();
}

template <class V>
cudaError_t launch_omega(const int64_t *ray_off, int64_t R, const uint32_t *vox, const float *t_in,
                         const float *t_out, const float *Zr, const V *T, double h, int8_t *result,
                         unsigned long long *counts, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    k_omega<V><<<nblk(R, 128), 128, 0, s>>>(ray_off, R, vox, t_in, t_out, Zr, T, h, result, counts);
    return cudaGetLastError();
}
template cudaError_t launch_omega<float>(const int64_t *, int64_t, const uint32_t *, const float *, const float *,
                                         const float *, const float *, double, int8_t *, unsigned long long *,
                                         cudaStream_t);
template cudaError_t launch_omega<double>(const int64_t *, int64_t, const uint32_t *, const float *, const float *,
                                          const float *, const double *, double, int8_t *, unsigned long long *,
                                          cudaStream_t);

int theta_grad_threads(int n_bins) {
    // whole warps, each thread a row of n_bins + 1 doubles: two warps while the
    // rows fit in 96 KB of shared memory, else one (up to 131 KB for 512 bins)
    return (size_t)64 * (n_bins + 1) * 8 <= 96 * 1024 ? 64 : 32;
}

cudaError_t launch_theta_grad(const ThetaTab &th, const int64_t *ray_off, int64_t R, const float *dmid,
                              const float *Zr, const double *gnu, double *part, int blocks, cudaStream_t s) {
    const int t = theta_grad_threads(th.n_bins);
    const size_t sm = (size_t)t * (th.n_bins + 1) * 8;
    if (sm > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_theta_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_theta_grad<<<(unsigned)blocks, (unsigned)t, sm, s>>>(th, ray_off, R, dmid, Zr, gnu, part);
    return cudaGetLastError();
}

void theta_far_setup(ThetaTab &th) {
    const int n = th.n_bins;
    // bound on the Gaussian density G: (1 - w) G below 2^-40 of the floor w / d_hi
    // (without an outlier term, below 1e-50, whose float is 0)
    const double floor_d = th.w > 0.0 ? th.w / th.dhi : 0.0;
    const double thr = th.w > 0.0 ? floor_d * std::ldexp(1.0, -40) / (1.0 - th.w) : 1e-50;
    // the likelihood of a far edge lies in [floor, floor (1 + 2^-40)]: its float is
    // the floor's when both ends round alike
    th.nu_far = (float)floor_d;
    th.far_ok = (float)(floor_d * (1.0 + std::ldexp(1.0, -40))) == th.nu_far;
    const double lthr = std::log(thr), c0 = 0.91893853320467274178;   // log sqrt(2 pi)
    // between nodes k and k + 1: G < thr once |Z - d - b| / sigma_max > sqrt(q),
    // q = 2 (-log thr - log sigma_min - log sqrt(2 pi))
    double pair[kMaxBins];
    for (int k = 0; k + 1 < n; ++k) {
        const double lo = std::fmin(th.ls[k], th.ls[k + 1]), hi = std::fmax(th.ls[k], th.ls[k + 1]);
        const double q = std::fmax(0.0, 2.0 * (-lthr - lo - c0));
        const double b = th.has_bias ? std::fmax(std::fabs((double)th.bias[k]), std::fabs((double)th.bias[k + 1])) : 0.0;
        pair[k] = b + std::exp(hi) * std::sqrt(q);
    }
    for (int k = 0; k + 1 < n; ++k) {
        double m = pair[k];
        if (k > 0) m = std::fmax(m, pair[k - 1]);
        if (k + 2 < n) m = std::fmax(m, pair[k + 1]);
        th.far_d[k] = (float)(m * (1.0 + 1e-6) + 1e-4);   // margin for the FP32 |Z - d| and bin
    }
    th.dlo_f = (float)th.dlo;
    th.inv_delta_f = (float)(1.0 / th.delta);
}

}  // namespace mrf
