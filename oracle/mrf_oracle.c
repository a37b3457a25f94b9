/*
 * mrf_oracle.c -- plain, slow, FP64 CPU oracle for ray-MRF loopy belief
 * propagation (MRFMap, arXiv 2006.03512).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the bench's
 * CPU-baseline / reference legs are the only users.  It shares no code, header
 * or constant with the CUDA library and neither side includes the other.
 *
 * What it computes, and where each step comes from:
 *
 *  1. Rays (Section III-A, "Ray Markov Random Field"; Section IV-A 3DDA
 *     traversal; Section IV-B 3-sigma truncation).  One ray per valid depth
 *     pixel, walked voxel by voxel with an Amanatides-Woo style traversal.  The
 *     walk follows a pinned FP32 recipe (written out in orc_ray_setup and
 *     orc_ray_walk) so that voxel indices and per-voxel depths are bit-exact
 *     with any other implementation of the same recipe.  Build with
 *     -ffp-contract=off: no fused multiply-add may change a rounding.
 *
 *  2. Sensor likelihood nu(d_i) (Eq. "noise": a Gaussian in the measured range
 *     with range-dependent sigma; Section IV-C: bias shifts the predicted
 *     mean), mixed with a uniform outlier floor w/d_hi.  FP64, log domain.
 *
 *  3. Ray-to-occupancy messages (Eqs. "pos" and "neg", with the visibility
 *     weighted depth message of Eq. "depth_message" as their summand), in FP64
 *     log domain, in the paper's order: P_i = prod_{k<i} mu(o_k=0),
 *     w_j = mu(o_j=1) nu(d_j) P_j, pos_i = sum_{j<i} w_j + nu(d_i) P_i,
 *     neg_i = sum_{j<i} w_j + (1/mu(o_i=0)) (sum_{j>i} w_j + nu_bg P_{N+1}).
 *     The nu_bg term is the all-empty configuration of the ray (reading: a
 *     background likelihood for "no voxel on the ray is occupied"; nu_bg = 0 is
 *     the paper taken literally).  A second, division-free form (the
 *     supplement's expansion with prod_{k<j, k!=i}) is kept for cross-checks.
 *
 *  4. Occupancy-to-ray messages (Eq. "node_to_factor": the prior factor times
 *     every other incoming ray message) and marginals (Eq. for p(x), the
 *     product of all incoming factor messages), held as log-odds:
 *     T_v = logit(gamma) + sum_r lambda_{r->v}, cavity L = T_v - lambda_{r->v}.
 *
 *  5. Schedule (Section IV-A, "up and down passes"): flooding.  Iteration 1
 *     sends mu(o=1) = init_p on every edge; each later iteration forms every
 *     cavity from the previous iteration's messages, then replaces all ray
 *     messages at once.  Marginals come after the last pass.
 *
 *  6. Gradient of a held-out depth likelihood (section 6, not in the paper).
 *  7. The accuracy metric of Section "Evaluation Metric for Probabilistic
 *     Occupancy Maps" (section 7).
 *  8. The implementation's variants (Section "Belief Propagation" of the
 *     implementation): traversed-length weighting and per-keyframe average
 *     messages (section 8).
 *
 * Numbers are FP64 throughout except the traversal recipe, which is FP32 by
 * definition.  Ray messages are clamped to +-64 in log-odds (a reading: with
 * nu_bg = 0 a one-voxel ray has an infinite message).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LAM_CLAMP 64.0
#define ORC_LOG_2PI 1.8378770664093454835606594728112353

/* ------------------------------------------------------------------------ */
/* inputs                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    float res;
    float origin[3];
} orc_grid;

typedef struct {
    int W, H;
    float fx, fy, cx, cy;
    double pose[12]; /* camera-to-world 3x4 row-major [R | c] */
} orc_camera;

typedef struct {
    int n_bins;
    float d_lo, d_hi;
    const float *log_sigma; /* n_bins */
    float outlier_w;
    const float *bias;      /* n_bins or NULL */
} orc_lut;

/* per-ray result of the setup step (exported for tests) */
typedef struct {
    float o[3], k[3], inv[3];
    float t0, t1, Z;
    int32_t s[3], e[3];
    int32_t N;
} orc_ray;

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1. traversal -- pinned FP32 recipe                                       */
/* ------------------------------------------------------------------------ */

/* sigma used for the 3-sigma truncation: a float table sig_k = (float)exp(L_k)
 * interpolated linearly in sigma with the same bin rule as the likelihood. */
static float trunc_sigma(const orc_lut *lut, const float *sig_tab, float Z)
{
    const float dlo = lut->d_lo;
    const float inv_delta = (float)((double)lut->n_bins / ((double)lut->d_hi - (double)lut->d_lo));
    float x = (Z - dlo) * inv_delta - 0.5f;
    float fk = floorf(x);
    int k;
    if (!(fk >= 0.0f)) k = 0;
    else if (fk > (float)(lut->n_bins - 2)) k = lut->n_bins - 2;
    else k = (int)fk;
    float f = x - (float)k;
    if (f < 0.0f) f = 0.0f;
    if (f > 1.0f) f = 1.0f;
    float a = (1.0f - f) * sig_tab[k];
    float b = f * sig_tab[k + 1];
    return a + b;
}

static int clamp_floor(float x, int n)
{
    float f = floorf(x);
    if (!(f >= 0.0f)) return 0;
    if (f > (float)(n - 1)) return n - 1;
    return (int)f;
}

static void cam_consts(const orc_grid *g, const orc_camera *cam, float o[3], float R[9])
{
    for (int a = 0; a < 3; ++a) {
        o[a] = (float)((cam->pose[a * 4 + 3] - (double)g->origin[a]) / (double)g->res);
        for (int b = 0; b < 3; ++b) R[a * 3 + b] = (float)cam->pose[a * 4 + b];
    }
}

/* Ray set-up for pixel (u, v) with z-depth z.  Every operation is one IEEE
 * FP32 rounding in the order written.  trunc = 0 walks to the grid exit (the
 * evaluation metric of section 7) instead of 3 sigma past the measurement. */
static void ray_setup(const orc_grid *g, const orc_camera *cam, const orc_lut *lut, const float *sig_tab, int u,
                      int v, float z, int trunc, orc_ray *r)
{
    float o[3], R[9];
    cam_consts(g, cam, o, R);
    const int n[3] = {g->nx, g->ny, g->nz};
    const float h = g->res;
    memset(r, 0, sizeof(*r));
    int valid = (z > 0.0f) && isfinite(z);
    float a = ((float)u - cam->cx) / cam->fx;
    float b = ((float)v - cam->cy) / cam->fy;
    float aa = a * a;
    float bb = b * b;
    float len = sqrtf((aa + bb) + 1.0f);
    for (int q = 0; q < 3; ++q) {
        float ea = R[q * 3 + 0] * a;
        float eb = R[q * 3 + 1] * b;
        float e = (ea + eb) + R[q * 3 + 2];
        r->k[q] = (e / len) / h;
        r->o[q] = o[q];
    }
    r->Z = z * len;
    float t0 = 0.0f, tex = INFINITY;
    int ok = 1;
    for (int q = 0; q < 3; ++q) {
        if (r->k[q] != 0.0f) {
            float inv = 1.0f / r->k[q];
            float ta = (0.0f - o[q]) * inv;
            float tb = ((float)n[q] - o[q]) * inv;
            float lo = ta < tb ? ta : tb;
            float hi = ta < tb ? tb : ta;
            r->inv[q] = inv;
            if (lo > t0) t0 = lo;
            if (hi < tex) tex = hi;
        } else {
            r->inv[q] = 0.0f;
            if (!(o[q] >= 0.0f && o[q] < (float)n[q])) ok = 0;
        }
    }
    float sig = valid && trunc ? trunc_sigma(lut, sig_tab, r->Z) : 0.0f;
    float tt = r->Z + 3.0f * sig;
    float t1 = !trunc || tex < tt ? tex : tt;
    r->t0 = t0;
    r->t1 = t1;
    if (!(valid && ok && t0 < t1)) {
        r->N = 0;
        return;
    }
    int N = 1;
    for (int q = 0; q < 3; ++q) {
        float ps = o[q] + t0 * r->k[q];
        float pe = o[q] + t1 * r->k[q];
        int s = clamp_floor(ps, n[q]);
        int e = clamp_floor(pe, n[q]);
        if (r->k[q] > 0.0f) { if (e < s) e = s; }
        else if (r->k[q] < 0.0f) { if (e > s) e = s; }
        else e = s;
        r->s[q] = s;
        r->e[q] = e;
        N += e > s ? e - s : s - e;
    }
    r->N = N;
}

void orc_ray_setup_one(const orc_grid *g, const orc_camera *cam, const orc_lut *lut,
                       const float *sig_tab, int u, int v, float z, orc_ray *r)
{
    ray_setup(g, cam, lut, sig_tab, u, v, z, 1, r);
}

/* Walk one ray; writes N voxel indices (x fastest) and N depths (midpoint
 * ranges); t_in / t_out (optional) get each voxel's entry and exit range. */
static void ray_walk(const orc_grid *g, const orc_ray *r, uint32_t *vox, float *d, float *t_in, float *t_out)
{
    int c[3] = {r->s[0], r->s[1], r->s[2]};
    float tin = r->t0;
    for (int i = 0; i < r->N; ++i) {
        float tout;
        int best = -1;
        if (i == r->N - 1) {
            tout = r->t1;
        } else {
            float bt = 0.0f;
            for (int q = 0; q < 3; ++q) {
                if (c[q] == r->e[q]) continue;
                float bound = (float)(c[q] + (r->k[q] > 0.0f ? 1 : 0));
                float tm = (bound - r->o[q]) * r->inv[q];
                if (best < 0 || tm < bt) { best = q; bt = tm; }
            }
            float m = bt < r->t1 ? bt : r->t1;
            tout = m > tin ? m : tin;
        }
        float s = tin + tout;
        d[i] = 0.5f * s;
        if (t_in) t_in[i] = tin;
        if (t_out) t_out[i] = tout;
        vox[i] = (uint32_t)c[0] + (uint32_t)g->nx * ((uint32_t)c[1] + (uint32_t)g->ny * (uint32_t)c[2]);
        if (best >= 0) {
            c[best] += r->k[best] > 0.0f ? 1 : -1;
            tin = tout;
        }
    }
}

void orc_ray_walk(const orc_grid *g, const orc_ray *r, uint32_t *vox, float *d) { ray_walk(g, r, vox, d, NULL, NULL); }

static float *make_sig_tab(const orc_lut *lut)
{
    float *t = (float *)malloc(sizeof(float) * (size_t)lut->n_bins);
    for (int k = 0; k < lut->n_bins; ++k) t[k] = (float)exp((double)lut->log_sigma[k]);
    return t;
}

/* Set-up for every pixel of a frame (row-major, ray id = v*W + u). */
void orc_frame_setup(const orc_grid *g, const orc_camera *cam, const orc_lut *lut,
                     const float *depth, orc_ray *rays)
{
    float *sig = make_sig_tab(lut);
    const int W = cam->W, H = cam->H;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        int u = (int)(p % W), v = (int)(p / W);
        orc_ray_setup_one(g, cam, lut, sig, u, v, depth[p], &rays[p]);
    }
    free(sig);
}

/* Walk every ray of a frame into a CSR whose offsets the caller computed from
 * the rays' N (ray_off has R+1 entries, relative to the arrays passed). */
void orc_frame_walk(const orc_grid *g, int64_t R, const orc_ray *rays, const int64_t *ray_off,
                    uint32_t *vox, float *d)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < R; ++r)
        orc_ray_walk(g, &rays[r], vox + ray_off[r], d + ray_off[r]);
}

/* ------------------------------------------------------------------------ */
/* 2. sensor likelihood (FP64, log domain)                                  */
/* ------------------------------------------------------------------------ */
static double lse2(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b)));
}

/* piecewise-linear table lookup at range d (bin centres d_lo + (k+1/2) delta) */
static double lut_interp(const orc_lut *lut, const float *tab, double d)
{
    const double delta = ((double)lut->d_hi - (double)lut->d_lo) / lut->n_bins;
    double x = (d - (double)lut->d_lo) / delta - 0.5;
    double fk = floor(x);
    int k;
    if (!(fk >= 0.0)) k = 0;
    else if (fk > lut->n_bins - 2) k = lut->n_bins - 2;
    else k = (int)fk;
    double f = x - k;
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return (1.0 - f) * (double)tab[k] + f * (double)tab[k + 1];
}

double orc_log_sigma_at(const orc_lut *lut, double d) { return lut_interp(lut, lut->log_sigma, d); }

/* log nu(d | Z) = log[(1-w) N(Z; d + b(d), sigma(d)) + w / d_hi] */
double orc_log_nu(const orc_lut *lut, double d, double Z)
{
    const double ls = lut_interp(lut, lut->log_sigma, d);
    const double b = lut->bias ? lut_interp(lut, lut->bias, d) : 0.0;
    const double sig = exp(ls);
    const double zz = (Z - (d + b)) / sig;
    const double lg = -0.5 * zz * zz - ls - 0.5 * ORC_LOG_2PI;
    const double w = lut->outlier_w;
    if (w <= 0.0) return lg;
    return lse2(log1p(-w) + lg, log(w) - log((double)lut->d_hi));
}

/* log of the all-empty likelihood when it defaults to the outlier density:
 * log(w / d_hi) with the table's own (float) w and d_hi; -inf when w = 0. */
double orc_default_log_nu_bg(const orc_lut *lut)
{
    if (lut->outlier_w <= 0.0f) return -INFINITY;
    return log((double)lut->outlier_w) - log((double)lut->d_hi);
}

/* log nu for every edge; ray r owns edges ray_off[r]..ray_off[r+1]-1 and has range Z[r] */
void orc_log_nu_edges(const orc_lut *lut, int64_t R, const int64_t *ray_off, const float *Z,
                      const float *d, double *log_nu)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < R; ++r)
        for (int64_t e = ray_off[r]; e < ray_off[r + 1]; ++e)
            log_nu[e] = orc_log_nu(lut, (double)d[e], (double)Z[r]);
}

/* ------------------------------------------------------------------------ */
/* 3. ray -> occupancy messages (Eqs. pos / neg), FP64 log domain           */
/* ------------------------------------------------------------------------ */
static double softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }

static double clamp_lam(double x)
{
    if (x != x) return 0.0;
    if (x > ORC_LAM_CLAMP) return ORC_LAM_CLAMP;
    if (x < -ORC_LAM_CLAMP) return -ORC_LAM_CLAMP;
    return x;
}

/* One ray of N voxels.  L[i]: log-odds of the incoming occupancy->ray message
 * mu(o_i); log_nu[i]: log nu(d_i); log_nu_bg: log of the all-empty likelihood
 * (-inf for none).  Writes lam[i] = log mu_{psi->o_i}(1) - log mu_{psi->o_i}(0).
 * work must hold 4*(N+1) doubles. */
void orc_ray_messages(int N, const double *L, const double *log_nu, double log_nu_bg,
                      double *lam, double *work)
{
    double *logP = work;            /* logP[i] = log prod_{k<i} mu(o_k=0), i = 0..N   */
    double *logw = work + (N + 1);  /* log w_i = log mu(o_i=1) + log nu_i + log P_i   */
    double *logA = work + 2 * (N + 1); /* log sum_{j<i} w_j                          */
    double *logS = work + 3 * (N + 1); /* log (sum_{j>i} w_j + nu_bg P_N)            */
    logP[0] = 0.0;
    for (int i = 0; i < N; ++i) {
        const double lm0 = -softplus(L[i]);
        const double lm1 = -softplus(-L[i]);
        logw[i] = lm1 + log_nu[i] + logP[i];
        logP[i + 1] = logP[i] + lm0;
    }
    logA[0] = -INFINITY;
    for (int i = 1; i <= N; ++i) logA[i] = lse2(logA[i - 1], logw[i - 1]);
    /* logS[i] = log( sum_{j>i} w_j + nu_bg P_{N} ) with 0-based i */
    logS[N - 1] = log_nu_bg + logP[N];
    for (int i = N - 2; i >= 0; --i) logS[i] = lse2(logS[i + 1], logw[i + 1]);
    for (int i = 0; i < N; ++i) {
        const double lm0 = -softplus(L[i]);
        const double lpos = lse2(logA[i], log_nu[i] + logP[i]);
        const double lneg = lse2(logA[i], logS[i] - lm0);
        lam[i] = clamp_lam(lpos - lneg);
    }
}

/* Division-free form of Eq. "neg" (the supplement's expansion with the product
 * over k<j, k!=i written out), O(N^2); used only to cross-check the form above. */
void orc_ray_messages_divfree(int N, const double *L, const double *log_nu, double log_nu_bg,
                              double *lam)
{
    for (int i = 0; i < N; ++i) {
        double lpre = -INFINITY;   /* log sum_{j<i} w_j */
        double lP = 0.0;           /* log prod_{k<j} mu(o_k=0) as j advances */
        for (int j = 0; j < i; ++j) {
            lpre = lse2(lpre, -softplus(-L[j]) + log_nu[j] + lP);
            lP += -softplus(L[j]);
        }
        const double lPi = lP;
        const double lpos = lse2(lpre, log_nu[i] + lPi);
        /* sum over j>i of mu(o_j=1) nu_j prod_{k<j, k != i} mu(o_k=0), plus the
         * all-empty term nu_bg prod_{k != i} mu(o_k=0) */
        double lpost = -INFINITY;
        double lQ = lPi;           /* log prod_{k<j, k!=i} mu(o_k=0) */
        for (int j = i + 1; j < N; ++j) {
            lpost = lse2(lpost, -softplus(-L[j]) + log_nu[j] + lQ);
            lQ += -softplus(L[j]);
        }
        lpost = lse2(lpost, log_nu_bg + lQ);
        const double lneg = lse2(lpre, lpost);
        lam[i] = clamp_lam(lpos - lneg);
    }
}

/* ------------------------------------------------------------------------ */
/* 4-5. flooding loopy BP over all rays                                     */
/* ------------------------------------------------------------------------ */

/* Voxel-major view of the edges (stable by edge id): counting sort.  vstart has
 * V+1 entries, eid has E entries. */
void orc_transpose(int64_t E, const uint32_t *vox, int64_t V, int64_t *vstart, int64_t *eid)
{
    memset(vstart, 0, sizeof(int64_t) * (size_t)(V + 1));
    for (int64_t e = 0; e < E; ++e) vstart[(int64_t)vox[e] + 1]++;
    for (int64_t v = 0; v < V; ++v) vstart[v + 1] += vstart[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V + 1));
    memcpy(fill, vstart, sizeof(int64_t) * (size_t)(V + 1));
    for (int64_t e = 0; e < E; ++e) eid[fill[vox[e]]++] = e;
    free(fill);
}

/* T_v = logit(gamma) + sum of the messages into v, in edge-id order */
static void voxel_totals(int64_t V, const int64_t *vstart, const int64_t *eid, const double *lam,
                         double logit_prior, double *T)
{
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < V; ++v) {
        double s = logit_prior;
        for (int64_t k = vstart[v]; k < vstart[v + 1]; ++k) s += lam[eid[k]];
        T[v] = s;
    }
}

/*
 * Full inference.  Inputs: R rays in CSR (ray_off[R+1]) over E edges with
 * voxel ids vox[E] < V and log-likelihoods log_nu[E]; prior gamma; init_p, the
 * first occupancy->ray message on every edge; log_nu_bg; iters passes.
 * Outputs: lam[E] (last ray->voxel log-odds messages), T[V] (log-odds
 * marginals), p[V] = sigmoid(T).  Returns 0, or -1 on allocation failure.
 */
int orc_bp(int64_t R, const int64_t *ray_off, const uint32_t *vox, const double *log_nu, int64_t V,
           double prior, double init_p, double log_nu_bg, int iters,
           double *lam, double *T, double *p)
{
    const int64_t E = ray_off[R];
    const double logit_prior = log(prior) - log1p(-prior);
    const double L0 = log(init_p) - log1p(-init_p);
    int64_t *vstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V + 1));
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    double *lam_new = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    if (!vstart || !eid || !lam_new) { free(vstart); free(eid); free(lam_new); return -1; }
    orc_transpose(E, vox, V, vstart, eid);
    int64_t maxN = 0;
    for (int64_t r = 0; r < R; ++r) {
        int64_t n = ray_off[r + 1] - ray_off[r];
        if (n > maxN) maxN = n;
    }
    for (int64_t e = 0; e < E; ++e) lam[e] = 0.0;   /* uniform ray->voxel messages */
    for (int64_t v = 0; v < V; ++v) T[v] = logit_prior;
    for (int it = 0; it < iters; ++it) {
#pragma omp parallel
        {
            double *Lb = (double *)malloc(sizeof(double) * (size_t)(maxN + 1));
            double *wk = (double *)malloc(sizeof(double) * (size_t)(4 * (maxN + 1)));
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < R; ++r) {
                const int64_t e0 = ray_off[r];
                const int N = (int)(ray_off[r + 1] - e0);
                if (N == 0) continue;
                for (int i = 0; i < N; ++i)
                    Lb[i] = (it == 0) ? L0 : T[vox[e0 + i]] - lam[e0 + i];
                orc_ray_messages(N, Lb, log_nu + e0, log_nu_bg, lam_new + e0, wk);
            }
            free(Lb);
            free(wk);
        }
        memcpy(lam, lam_new, sizeof(double) * (size_t)E);
        voxel_totals(V, vstart, eid, lam, logit_prior, T);
    }
    for (int64_t v = 0; v < V; ++v) p[v] = 1.0 / (1.0 + exp(-T[v]));
    free(vstart);
    free(eid);
    free(lam_new);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 6. differentiation with respect to the noise table                       */
/* ------------------------------------------------------------------------ */
/*
 * Not in the paper: the gradient of a held-out depth likelihood with respect
 * to the sensor-noise table, for learning the table (the paper fits it
 * offline, Section IV-C).  The map's edges (which voxels each ray crosses,
 * their ranges d and the ray's measured range Z) are held fixed; the table
 * theta = (log sigma at the n_bins bin centres, outlier weight w) enters
 * through every edge's likelihood nu and through nu_bg = w / d_hi.
 *
 * Loss: for held-out rays r over voxels v_1..v_N with marginals p and
 * likelihoods nu_i, the probability of the measured depth when the occupancy
 * of each voxel is drawn independently from its marginal (Eq.
 * "depth_message" summed over the first occupied voxel, with mu = p):
 *   S_r = sum_i nu_i p_{v_i} Q_i + nu_bg Q_{N+1},   Q_i = prod_{k<i} (1 - p_{v_k}),
 *   loss = -sum_r log S_r.
 *
 * Everything here is FP64 and linear-domain; the forward BP is the same
 * flooding schedule as orc_bp (its messages come from orc_ray_messages).
 */

/* table position of range d: bin k and weight f of bin k+1 (the rule of lut_interp) */
static void lut_pos(const orc_lut *lut, double d, int *k_out, double *f_out)
{
    const double delta = ((double)lut->d_hi - (double)lut->d_lo) / lut->n_bins;
    double x = (d - (double)lut->d_lo) / delta - 0.5;
    double fk = floor(x);
    int k;
    if (!(fk >= 0.0)) k = 0;
    else if (fk > lut->n_bins - 2) k = lut->n_bins - 2;
    else k = (int)fk;
    double f = x - k;
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    *k_out = k;
    *f_out = f;
}

/* nu(d | Z; theta) = (1 - w) N(Z; d + b(d), sigma(d)) + w / d_hi with log sigma
 * interpolated from ls_tab (FP64 table values), and its partial derivatives
 * with respect to log sigma(d) and w. */
static double nu_theta(const orc_lut *lut, const double *ls_tab, double w, double d, double Z,
                       int *k, double *f, double *dnu_dls, double *dnu_dw)
{
    lut_pos(lut, d, k, f);
    const double ls = (1.0 - *f) * ls_tab[*k] + *f * ls_tab[*k + 1];
    const double b = lut->bias ? (1.0 - *f) * (double)lut->bias[*k] + *f * (double)lut->bias[*k + 1] : 0.0;
    const double zz = (Z - (d + b)) / exp(ls);
    const double G = exp(-0.5 * zz * zz - ls - 0.5 * ORC_LOG_2PI);
    if (dnu_dls) *dnu_dls = (1.0 - w) * G * (zz * zz - 1.0);
    if (dnu_dw) *dnu_dw = -G + 1.0 / (double)lut->d_hi;
    return (1.0 - w) * G + w / (double)lut->d_hi;
}

void orc_nu_theta_edges(const orc_lut *lut, const double *ls_tab, double w, int64_t R, const int64_t *ray_off,
                        const float *Z, const float *d, double *nu)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < R; ++r)
        for (int64_t e = ray_off[r]; e < ray_off[r + 1]; ++e) {
            int k;
            double f;
            nu[e] = nu_theta(lut, ls_tab, w, (double)d[e], (double)Z[r], &k, &f, NULL, NULL);
        }
}

/* Held-out loss (definition above).  When the gradient pointers are non-NULL,
 * adds d loss / d p_v into gp[V], d loss / d nu_e into gnu[E] and d loss /
 * d nu_bg into *gnu_bg.  Rays are visited in order, so every sum has a fixed
 * order. */
double orc_heldout_loss(int64_t R, const int64_t *ray_off, const uint32_t *vox, const double *nu, double nu_bg,
                        const double *p, double *gp, double *gnu, double *gnu_bg)
{
    double loss = 0.0;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t e0 = ray_off[r], e1 = ray_off[r + 1];
        if (e1 == e0) continue;
        /* S = sum_i nu_i p_i Q_i + nu_bg Q_{N+1} */
        double S = 0.0, Q = 1.0;
        for (int64_t e = e0; e < e1; ++e) {
            const double pv = p[vox[e]];
            S += nu[e] * pv * Q;
            Q *= 1.0 - pv;
        }
        S += nu_bg * Q;
        loss -= log(S);
        if (!gp) continue;
        /* dS/dp_i = Q_i (nu_i - R_i), R_i = sum_{j>i} nu_j p_j prod_{i<k<j}(1-p_k) + nu_bg prod_{k>i}(1-p_k);
         * dS/dnu_i = p_i Q_i; dS/dnu_bg = Q_{N+1} */
        const double gS = -1.0 / S;
        if (gnu_bg) *gnu_bg += gS * Q;
        double Rs = nu_bg;   /* R_i for the voxel being visited, backwards */
        /* Q_i going backwards: Q_i = Q_{i+1} / (1 - p_i) is not safe when p_i = 1,
         * so the prefix products are recomputed forwards per ray */
        double *Qs = (double *)malloc(sizeof(double) * (size_t)(e1 - e0));
        double q = 1.0;
        for (int64_t e = e0; e < e1; ++e) {
            Qs[e - e0] = q;
            q *= 1.0 - p[vox[e]];
        }
        for (int64_t e = e1 - 1; e >= e0; --e) {
            const double pv = p[vox[e]];
            const double Qi = Qs[e - e0];
            gp[vox[e]] += gS * Qi * (nu[e] - Rs);
            if (gnu) gnu[e] += gS * pv * Qi;
            Rs = nu[e] * pv + (1.0 - pv) * Rs;
        }
        free(Qs);
    }
    return loss;
}

/* Adjoint of orc_ray_messages for one ray, restated in the linear domain:
 * P_0 = 1, P_{i+1} = P_i m0_i; A_0 = 0, A_{i+1} = A_i + P_i m1_i nu_i;
 * B_{N-1} = nu_bg, B_{i-1} = m1_i nu_i + m0_i B_i; pos_i = A_i + P_i nu_i,
 * neg_i = A_i + P_i B_i, lam_i = log(pos_i / neg_i) (Eqs. "pos"/"neg" with the
 * 1/mu(o_i=0) cancelled).  Given g[i] = d loss / d lam_i, writes gL[i] =
 * d loss / d L_i and adds d loss / d nu_i into gnu[i] and d loss / d nu_bg into
 * *gnu_bg.  A message the forward clamps to +-64 passes no gradient.  work
 * must hold 9 * (N + 1) doubles. */
void orc_ray_messages_adjoint(int N, const double *L, const double *nu, double nu_bg, const double *g,
                              double *gL, double *gnu, double *gnu_bg, double *work)
{
    double *m1 = work, *m0 = work + (N + 1), *P = work + 2 * (N + 1), *A = work + 3 * (N + 1);
    double *B = work + 4 * (N + 1), *gpos = work + 5 * (N + 1), *gneg = work + 6 * (N + 1);
    double *gm1 = work + 7 * (N + 1), *gm0 = work + 8 * (N + 1);
    for (int i = 0; i < N; ++i) {
        m1[i] = 1.0 / (1.0 + exp(-L[i]));
        m0[i] = 1.0 / (1.0 + exp(L[i]));
        gm1[i] = gm0[i] = 0.0;
    }
    P[0] = 1.0;
    A[0] = 0.0;
    for (int i = 0; i < N; ++i) {
        P[i + 1] = P[i] * m0[i];
        A[i + 1] = A[i] + P[i] * m1[i] * nu[i];
    }
    B[N - 1] = nu_bg;
    for (int i = N - 1; i >= 1; --i) B[i - 1] = m1[i] * nu[i] + m0[i] * B[i];
    for (int i = 0; i < N; ++i) {
        const double pos = A[i] + P[i] * nu[i], neg = A[i] + P[i] * B[i];
        const double lam = log(pos) - log(neg);
        const int live = lam == lam && fabs(lam) < ORC_LAM_CLAMP;
        gpos[i] = live ? g[i] / pos : 0.0;
        gneg[i] = live ? -g[i] / neg : 0.0;
    }
    /* forward quantities A and P, in reverse */
    double gA = 0.0, gP = 0.0;   /* adjoints of A_{i+1}, P_{i+1} */
    for (int i = N - 1; i >= 0; --i) {
        /* A_{i+1} = A_i + P_i m1_i nu_i;  P_{i+1} = P_i m0_i */
        gm1[i] += gA * P[i] * nu[i];
        gnu[i] += gA * P[i] * m1[i];
        gm0[i] += gP * P[i];
        const double gPi = gpos[i] * nu[i] + gneg[i] * B[i] + gA * m1[i] * nu[i] + gP * m0[i];
        const double gAi = gpos[i] + gneg[i] + gA;
        gnu[i] += gpos[i] * P[i];
        gA = gAi;
        gP = gPi;
    }
    /* backward quantity B, forwards: B_{i-1} = m1_i nu_i + m0_i B_i */
    double gB = 0.0;   /* adjoint of B_{i-1} carried to step i */
    for (int i = 0; i < N; ++i) {
        if (i >= 1) {
            gm1[i] += gB * nu[i];
            gnu[i] += gB * m1[i];
            gm0[i] += gB * B[i];
        }
        gB = gneg[i] * P[i] + (i >= 1 ? gB * m0[i] : 0.0);
    }
    *gnu_bg += gB;   /* B_{N-1} = nu_bg */
    for (int i = 0; i < N; ++i) gL[i] = (gm1[i] - gm0[i]) * m1[i] * m0[i];
}

/*
 * Loss and gradient.  Training edges: R rays in CSR over vox, ranges d and
 * per-ray Z; held-out rays likewise (Rh, ...).  theta: ls_tab[n_bins] (FP64
 * log sigma at the bin centres; lut supplies n_bins, d_lo, d_hi and bias) and
 * w.  nu_bg = w / d_hi.  BP: prior, init_p, iters passes (the schedule of
 * orc_bp).  Writes *loss; when g_ls is non-NULL also g_ls[n_bins] and *g_w.
 * The forward keeps every pass's messages and voxel totals; the reverse pass
 * walks the passes back, recomputing each pass's cavities from them.
 * Returns 0, or -1 on allocation failure.
 */
int orc_grad(const orc_lut *lut, const double *ls_tab, double w, int64_t R, const int64_t *ray_off,
             const uint32_t *vox, const float *d, const float *Z, int64_t Rh, const int64_t *ray_off_h,
             const uint32_t *vox_h, const float *d_h, const float *Z_h, int64_t V, double prior, double init_p,
             int iters, double *loss, double *g_ls, double *g_w)
{
    const int64_t E = ray_off[R], Eh = ray_off_h[Rh];
    const int K = iters;
    const double logit_prior = log(prior) - log1p(-prior);
    const double L0 = log(init_p) - log1p(-init_p);
    const double nu_bg = w / (double)lut->d_hi;
    const size_t E1 = (size_t)(E > 0 ? E : 1), Eh1 = (size_t)(Eh > 0 ? Eh : 1);
    double *nu = (double *)malloc(sizeof(double) * E1);
    double *lnu = (double *)malloc(sizeof(double) * E1);
    double *nuh = (double *)malloc(sizeof(double) * Eh1);
    double *lam_ck = (double *)malloc(sizeof(double) * E1 * (size_t)(K + 1));
    double *T_ck = (double *)malloc(sizeof(double) * (size_t)V * (size_t)(K + 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)V);
    int64_t *vstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V + 1));
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * E1);
    if (!nu || !lnu || !nuh || !lam_ck || !T_ck || !p || !vstart || !eid) {
        free(nu); free(lnu); free(nuh); free(lam_ck); free(T_ck); free(p); free(vstart); free(eid);
        return -1;
    }
    orc_nu_theta_edges(lut, ls_tab, w, R, ray_off, Z, d, nu);
    orc_nu_theta_edges(lut, ls_tab, w, Rh, ray_off_h, Z_h, d_h, nuh);
    for (int64_t e = 0; e < E; ++e) lnu[e] = log(nu[e]);
    orc_transpose(E, vox, V, vstart, eid);
    int64_t maxN = 1;
    for (int64_t r = 0; r < R; ++r)
        if (ray_off[r + 1] - ray_off[r] > maxN) maxN = ray_off[r + 1] - ray_off[r];
    const double lbg = w > 0.0 ? log(nu_bg) : -INFINITY;

    /* forward: pass t reads lam_ck[t-1], T_ck[t-1] and writes lam_ck[t], T_ck[t] */
    for (int64_t e = 0; e < E; ++e) lam_ck[e] = 0.0;
    for (int64_t v = 0; v < V; ++v) T_ck[v] = logit_prior;
    for (int t = 1; t <= K; ++t) {
        const double *lp_ = lam_ck + (size_t)(t - 1) * E1;
        const double *Tp = T_ck + (size_t)(t - 1) * V;
        double *ln_ = lam_ck + (size_t)t * E1;
#pragma omp parallel
        {
            double *Lb = (double *)malloc(sizeof(double) * (size_t)(maxN + 1));
            double *wk = (double *)malloc(sizeof(double) * (size_t)(4 * (maxN + 1)));
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < R; ++r) {
                const int64_t e0 = ray_off[r];
                const int N = (int)(ray_off[r + 1] - e0);
                if (N == 0) continue;
                for (int i = 0; i < N; ++i) Lb[i] = (t == 1) ? L0 : Tp[vox[e0 + i]] - lp_[e0 + i];
                orc_ray_messages(N, Lb, lnu + e0, lbg, ln_ + e0, wk);
            }
            free(Lb);
            free(wk);
        }
        voxel_totals(V, vstart, eid, ln_, logit_prior, T_ck + (size_t)t * V);
    }
    const double *TK = T_ck + (size_t)K * V;
    for (int64_t v = 0; v < V; ++v) p[v] = 1.0 / (1.0 + exp(-TK[v]));

    int rc = 0;
    if (!g_ls) {
        *loss = orc_heldout_loss(Rh, ray_off_h, vox_h, nuh, nu_bg, p, NULL, NULL, NULL);
    } else {
        double *gT = (double *)calloc((size_t)V, sizeof(double));
        double *gLn = (double *)calloc(E1, sizeof(double));    /* d loss / d L^(t+1) */
        double *gLc = (double *)calloc(E1, sizeof(double));    /* d loss / d L^(t) */
        double *gnu = (double *)calloc(E1, sizeof(double));
        double *gnuh = (double *)calloc(Eh1, sizeof(double));
        double *gbg_r = (double *)calloc((size_t)(R > 0 ? R : 1), sizeof(double));
        double gbg = 0.0;
        if (!gT || !gLn || !gLc || !gnu || !gnuh || !gbg_r) {
            rc = -1;
        } else {
            /* held-out loss, then through p = sigmoid(T^K) */
            *loss = orc_heldout_loss(Rh, ray_off_h, vox_h, nuh, nu_bg, p, gT, gnuh, &gbg);
            for (int64_t v = 0; v < V; ++v) gT[v] *= p[v] * (1.0 - p[v]);
            for (int t = K; t >= 1; --t) {
                const double *lp_ = lam_ck + (size_t)(t - 1) * E1;
                const double *Tp = T_ck + (size_t)(t - 1) * V;
#pragma omp parallel
                {
                    double *Lb = (double *)malloc(sizeof(double) * (size_t)(maxN + 1));
                    double *gl = (double *)malloc(sizeof(double) * (size_t)(maxN + 1));
                    double *wk = (double *)malloc(sizeof(double) * (size_t)(9 * (maxN + 1)));
#pragma omp for schedule(dynamic, 256)
                    for (int64_t r = 0; r < R; ++r) {
                        const int64_t e0 = ray_off[r];
                        const int N = (int)(ray_off[r + 1] - e0);
                        if (N == 0) continue;
                        /* T^(t) = logit gamma + sum lam^(t); L^(t+1) = T^(t)[v] - lam^(t) */
                        for (int i = 0; i < N; ++i) {
                            gl[i] = gT[vox[e0 + i]] - gLn[e0 + i];
                            Lb[i] = (t == 1) ? L0 : Tp[vox[e0 + i]] - lp_[e0 + i];
                        }
                        double gb = 0.0;
                        orc_ray_messages_adjoint(N, Lb, nu + e0, nu_bg, gl, gLc + e0, gnu + e0, &gb, wk);
                        gbg_r[r] += gb;
                    }
                    free(Lb);
                    free(gl);
                    free(wk);
                }
                /* d loss / d T^(t-1)[v] = sum over the voxel's edges of d loss / d L^(t) */
                if (t >= 2) voxel_totals(V, vstart, eid, gLc, 0.0, gT);
                double *sw = gLn;
                gLn = gLc;
                gLc = sw;
            }
            for (int64_t r = 0; r < R; ++r) gbg += gbg_r[r];
            /* theta: through every edge's nu and through nu_bg = w / d_hi */
            for (int k = 0; k < lut->n_bins; ++k) g_ls[k] = 0.0;
            double gw = gbg / (double)lut->d_hi;
            for (int pass = 0; pass < 2; ++pass) {
                const int64_t RR = pass ? Rh : R;
                const int64_t *ro = pass ? ray_off_h : ray_off;
                const float *dd = pass ? d_h : d, *ZZ = pass ? Z_h : Z;
                const double *gn = pass ? gnuh : gnu;
                for (int64_t r = 0; r < RR; ++r)
                    for (int64_t e = ro[r]; e < ro[r + 1]; ++e) {
                        int k;
                        double f, dls, dw;
                        nu_theta(lut, ls_tab, w, (double)dd[e], (double)ZZ[r], &k, &f, &dls, &dw);
                        g_ls[k] += gn[e] * dls * (1.0 - f);
                        g_ls[k + 1] += gn[e] * dls * f;
                        gw += gn[e] * dw;
                    }
            }
            *g_w = gw;
        }
        free(gT); free(gLn); free(gLc); free(gnu); free(gnuh); free(gbg_r);
    }
    free(nu); free(lnu); free(nuh); free(lam_ck); free(T_ck); free(p); free(vstart); free(eid);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 7. the evaluation metric of Section "Evaluation Metric for Probabilistic */
/*    Occupancy Maps"                                                       */
/* ------------------------------------------------------------------------ */
/*
 * A ray, walked to the map boundary, crosses voxel i over [s_i, s_i + l_i).
 * Readings (the paper gives alpha only as a piecewise-constant occlusion
 * density): alpha_i = -log(1 - p_i) / h, so that a ray crossing a whole voxel
 * keeps visibility 1 - p_i; vis_0 = 1, vis_{i+1} = vis_i exp(-alpha_i l_i);
 * omega(s) = alpha(s) vis(s) is largest, inside each voxel, at its entry, so
 * the most likely generating surface is the voxel with the largest
 * alpha_i vis_i (the first one on ties).  At the map boundary the remaining
 * visibility vis_N is the chance the surface lies beyond the map; when it
 * exceeds that voxel's occlusion mass vis_i - vis_{i+1}, the surface is taken
 * to be beyond the boundary.  The ray is accurately classified when its
 * measured range Z lies in [s_i, s_i + l_i) of the chosen voxel, or, beyond
 * the boundary, when Z > s_N (the range at which it leaves the map).
 * Returns 1 (accurate), 0 (not), with the voxel chosen in *chosen (-1 beyond).
 */
int orc_omega_ray(int N, const uint32_t *vox, const float *t_in, const float *t_out, const double *p, double h,
                  float Z, int *chosen)
{
    double vis = 1.0, best_w = -1.0, best_mass = 0.0;
    int best = -1;
    for (int i = 0; i < N; ++i) {
        const double pi = p[vox[i]];
        const double l = (double)t_out[i] - (double)t_in[i];
        const double a = pi >= 1.0 ? INFINITY : -log1p(-pi) / h;
        const double w = a * vis;   /* a = inf with vis = 0 is NaN: never a maximum */
        const double vnext = pi >= 1.0 ? (l > 0.0 ? 0.0 : vis) : vis * exp(-a * l);
        if (w > best_w) {
            best_w = w;
            best = i;
            best_mass = vis - vnext;
        }
        vis = vnext;
    }
    if (best < 0 || vis > best_mass) {
        *chosen = -1;
        return N > 0 && Z > t_out[N - 1];
    }
    *chosen = best;
    return t_in[best] <= Z && Z < t_out[best];
}

/* Every pixel of a frame with a valid depth and a non-empty walk to the grid
 * exit: result[pixel] = 1 accurate, 0 not, -1 not evaluated.  p: marginals of
 * the nx*ny*nz voxels (x fastest).  Returns the number evaluated. */
int64_t orc_omega_frame(const orc_grid *g, const orc_camera *cam, const orc_lut *lut, const float *depth,
                        const double *p, int8_t *result)
{
    const int64_t npix = (int64_t)cam->W * cam->H;
    float *sig_tab = make_sig_tab(lut);
    int64_t n = 0;
#pragma omp parallel reduction(+ : n)
    {
        int cap = 1024;
        uint32_t *vox = (uint32_t *)malloc(sizeof(uint32_t) * cap);
        float *d = (float *)malloc(sizeof(float) * cap), *ti = (float *)malloc(sizeof(float) * cap),
              *to = (float *)malloc(sizeof(float) * cap);
#pragma omp for schedule(dynamic, 256)
        for (int64_t px = 0; px < npix; ++px) {
            orc_ray r;
            ray_setup(g, cam, lut, sig_tab, (int)(px % cam->W), (int)(px / cam->W), depth[px], 0, &r);
            if (r.N <= 0) {
                result[px] = -1;
                continue;
            }
            if (r.N > cap) {
                cap = r.N;
                vox = (uint32_t *)realloc(vox, sizeof(uint32_t) * cap);
                d = (float *)realloc(d, sizeof(float) * cap);
                ti = (float *)realloc(ti, sizeof(float) * cap);
                to = (float *)realloc(to, sizeof(float) * cap);
            }
            ray_walk(g, &r, vox, d, ti, to);
            int chosen;
            result[px] = (int8_t)orc_omega_ray(r.N, vox, ti, to, p, (double)g->res, r.Z, &chosen);
            n += 1;
        }
        free(vox); free(d); free(ti); free(to);
    }
    free(sig_tab);
    return n;
}

/* ------------------------------------------------------------------------ */
/* 8. the paper's implementation variants (Section "Belief Propagation"    */
/*    of the implementation)                                                */
/* ------------------------------------------------------------------------ */
/*
 * Two departures from exact flooding BP that the paper's implementation makes.
 *
 * Traversed-length weighting.  The paper weighs each ray's contribution to a
 * voxel by the length the ray travels inside it, without saying how.
 * Reading: the ray->voxel log-odds message lambda_e enters the voxel's belief
 * as w_e lambda_e, w_e = min(1, l_e / h) with l_e the traversed length and h
 * the voxel edge (a ray crossing a whole voxel counts fully, one that clips a
 * corner or stops inside it counts in proportion); the voxel->ray message a
 * ray receives leaves out its own weighted contribution:
 *   T_v = logit gamma + sum_e w_e lambda_e,   L_e = T_v - w_e lambda_e.
 * The ray factor itself is unchanged.
 *
 * Per-keyframe average messages.  All rays of one keyframe through a voxel
 * are taken to send the same message, the average of theirs; the voxel->ray
 * message then leaves out that average:
 *   s_e = w_e lambda_e,  sbar_{f,v} = mean of s_e over frame f's edges into v,
 *   T_v = logit gamma + sum_e s_e,  L_e = T_v - sbar_{f(e),v}.
 * (sum_e s_e = sum_f n_{f,v} sbar_{f,v}: the belief is unchanged.)
 *
 * wlen (E entries) or ray_frame (R entries, non-decreasing: rays frame-major)
 * may be NULL, which turns the variant off.  lam receives the stored
 * per-edge values the next pass would subtract (w_e lambda_e, averaged per
 * (frame, voxel) when averaging).  Returns 0, -1 on allocation failure, -2
 * when ray_frame decreases.
 */
int orc_bp_variants(int64_t R, const int64_t *ray_off, const uint32_t *vox, const double *log_nu, int64_t V,
                    double prior, double init_p, double log_nu_bg, int iters, const double *wlen,
                    const int32_t *ray_frame, double *lam, double *T, double *p)
{
    const int64_t E = ray_off[R];
    const double logit_prior = log(prior) - log1p(-prior);
    const double L0 = log(init_p) - log1p(-init_p);
    for (int64_t r = 1; ray_frame && r < R; ++r)
        if (ray_frame[r] < ray_frame[r - 1]) return -2;
    int64_t *vstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V + 1));
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    double *lam_new = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    int32_t *edge_frame = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    if (!vstart || !eid || !lam_new || !edge_frame) {
        free(vstart); free(eid); free(lam_new); free(edge_frame);
        return -1;
    }
    orc_transpose(E, vox, V, vstart, eid);   /* each voxel's edges in increasing edge order */
    int64_t maxN = 0;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t n = ray_off[r + 1] - ray_off[r];
        if (n > maxN) maxN = n;
        for (int64_t e = ray_off[r]; e < ray_off[r + 1]; ++e) edge_frame[e] = ray_frame ? ray_frame[r] : 0;
    }
    for (int64_t e = 0; e < E; ++e) lam[e] = 0.0;
    for (int64_t v = 0; v < V; ++v) T[v] = logit_prior;
    for (int it = 0; it < iters; ++it) {
        /* ray -> voxel messages from the cavities of the previous pass */
#pragma omp parallel
        {
            double *Lb = (double *)malloc(sizeof(double) * (size_t)(maxN + 1));
            double *wk = (double *)malloc(sizeof(double) * (size_t)(4 * (maxN + 1)));
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < R; ++r) {
                const int64_t e0 = ray_off[r];
                const int N = (int)(ray_off[r + 1] - e0);
                if (N == 0) continue;
                for (int i = 0; i < N; ++i) Lb[i] = (it == 0) ? L0 : T[vox[e0 + i]] - lam[e0 + i];
                orc_ray_messages(N, Lb, log_nu + e0, log_nu_bg, lam_new + e0, wk);
            }
            free(Lb);
            free(wk);
        }
        /* weighted contributions and the voxel beliefs */
        for (int64_t e = 0; e < E; ++e) lam[e] = wlen ? wlen[e] * lam_new[e] : lam_new[e];
        voxel_totals(V, vstart, eid, lam, logit_prior, T);
        /* one average per (keyframe, voxel): within a voxel's edge list the
         * edges of one frame are contiguous (rays are frame-major) */
        if (ray_frame) {
#pragma omp parallel for schedule(dynamic, 4096)
            for (int64_t v = 0; v < V; ++v) {
                int64_t a = vstart[v];
                while (a < vstart[v + 1]) {
                    int64_t b = a + 1;
                    while (b < vstart[v + 1] && edge_frame[eid[b]] == edge_frame[eid[a]]) ++b;
                    double s = 0.0;
                    for (int64_t k = a; k < b; ++k) s += lam[eid[k]];
                    const double mean = s / (double)(b - a);
                    for (int64_t k = a; k < b; ++k) lam[eid[k]] = mean;
                    a = b;
                }
            }
        }
    }
    for (int64_t v = 0; v < V; ++v) p[v] = 1.0 / (1.0 + exp(-T[v]));
    free(vstart);
    free(eid);
    free(lam_new);
    free(edge_frame);
    return 0;
}

/* The walk of a frame with each voxel's entry and exit ranges (metres). */
void orc_frame_walk_seg(const orc_grid *g, int64_t R, const orc_ray *rays, const int64_t *ray_off,
                        uint32_t *vox, float *d, float *t_in, float *t_out)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < R; ++r)
        ray_walk(g, &rays[r], vox + ray_off[r], d + ray_off[r], t_in + ray_off[r], t_out + ray_off[r]);
}
