"""Whole-BP parity bars for the GPU tests (test helper; imports only the oracle).

Loopy BP has no contraction guarantee (Section III-B), so how closely an FP32
implementation can follow the FP64 oracle after many passes depends on the
map.  The bar is therefore tied to the oracle's own measured sensitivity to the
two inputs an FP32 implementation must round: the oracle is run again with 1e-7
relative noise on its likelihoods, and again with its first-pass message moved
by one float32 ulp of its log-odds (a change that reaches every edge at once);
d = the larger |p_probe - p_oracle| per voxel.
  * s = max d <= 5e-6 (well-conditioned): 1e-4 on every voxel, the FP32 bar;
  * otherwise 99.9% of voxels within max(1e-5, 100 * p99.9(d)) and every voxel
    within max(1e-4, 100 * s): rounding moves voxels by at most about what the
    probe moved them, with a factor 100 for the different directions FP32
    rounding and a single random probe take.
"""
import numpy as np

import oracle

P_TOL = 1e-4
WELL_CONDITIONED = 5e-6


def init_ulp(init_p):
    """The first-pass message whose log-odds is one float32 ulp above init_p's."""
    L0 = np.log(init_p) - np.log1p(-init_p)
    L1 = L0 + float(np.spacing(np.float32(abs(L0)))) if L0 != 0 else 0.0
    return float(1.0 / (1.0 + np.exp(-L1)))


def sensitivity_map(ray_off, vox, log_nu, V, prior, init_p, log_nu_bg, iters, p_ref, bp=None, extra=(), seed=0):
    """|dp| per voxel of the oracle's BP under rounding-size changes of its inputs: 1e-7 relative
    noise on its likelihoods, and (where the first-pass log-odds is not 0, which float32 holds
    exactly) that log-odds moved by one float32 ulp; the larger of the two per voxel."""
    bp = oracle.bp if bp is None else bp
    rng = np.random.default_rng(seed)
    noisy = log_nu + rng.normal(0, 1e-7, len(log_nu))
    d = np.abs(bp(ray_off, vox, noisy, V, prior, init_p, log_nu_bg, iters, *extra)[2] - p_ref)
    ip1 = init_ulp(init_p)
    if ip1 != init_p:
        d = np.maximum(d, np.abs(bp(ray_off, vox, log_nu, V, prior, ip1, log_nu_bg, iters, *extra)[2] - p_ref))
    return d


def workload_sensitivity(w, ref, init_p=None, log_nu_bg=None):
    """sensitivity_map for oracle.infer(w, ...) output ref."""
    lbg = oracle.default_log_nu_bg(w.lut) if log_nu_bg is None else log_nu_bg
    ip = w.prior if init_p is None else init_p
    return sensitivity_map(ref["csr"]["ray_off"], ref["csr"]["vox"], ref["log_nu"], w.grid.n_voxels, w.prior, ip,
                           lbg, w.iters, ref["p"])


def check_marginals(p, p_ref, sens, what=""):
    """Asserts the bar above for GPU marginals p against oracle marginals p_ref; returns |p - p_ref|."""
    p = np.asarray(p, np.float64).ravel()
    err = np.abs(p - p_ref)
    assert np.all((p >= 0) & (p <= 1)), what
    s = float(sens.max())
    if s <= WELL_CONDITIONED:
        assert err.max() <= P_TOL, (what, float(err.max()), s)
    else:
        q = float(np.percentile(err, 99.9))
        assert q <= max(1e-5, 100 * float(np.percentile(sens, 99.9))), (what, q, s)
        assert err.max() <= max(P_TOL, 100 * s), (what, float(err.max()), s)
    return err
