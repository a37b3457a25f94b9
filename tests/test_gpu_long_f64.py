"""FP64 accumulations for long rays in an FP32 context (mrf_options.long_ray_f64).

Rays longer than the threshold get their messages from FP64 prefix and suffix recurrences over the same
FP32 cavities and likelihoods; stored as FP32 they must equal the FP64 oracle's messages from the GPU's own
previous state to FP32 rounding, a bar 20x tighter than the FP32 kernels' (2e-5).  With a threshold above
every ray the path is the ungrouped FP32 one, bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as m
    m.build()
    return m


def gpu_map(m, w, **opt):
    mp = m.Map(w.grid, w.prior, m.Options(**opt))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    return mp


@pytest.mark.parametrize("thr", [8, 30])
def test_long_ray_messages_are_fp64_accurate(m, thr):
    w = make_workload("room_small")
    ref = oracle.trace_frames(w.grid, w.frames, w.lut)
    ro, vox = ref["ray_off"], ref["vox"].astype(np.int64)
    n = np.diff(ro)
    mp = gpu_map(m, w, long_ray_f64=thr)
    mp.infer(0)
    nu = mp.export_nu().cpu().numpy().astype(np.float64)
    lbg = oracle.default_log_nu_bg(w.lut)
    L0 = np.float64(np.float32(0.0))       # first pass: cavity logit(prior) - logit(prior) = 0 for init = prior
    lam_prev = T_prev = None
    long_rays = np.flatnonzero(n > thr)
    assert len(long_rays) > 100
    for t in range(1, 4):
        mp.infer(t)
        lam32, T32 = (x.cpu().numpy() for x in mp.export_messages())
        lam = lam32.astype(np.float64)
        L = np.full(len(vox), L0) if t == 1 else (T_prev[vox] - lam_prev).astype(np.float64)
        worst_long = worst_short = 0.0
        for r in range(len(ro) - 1):
            a, b = ro[r], ro[r + 1]
            if b == a:
                continue
            lr = oracle.ray_messages(L[a:b], np.log(nu[a:b]), lbg)
            err = float(np.max(np.abs(lam[a:b] - lr) / (1 + np.abs(lr))))
            if b - a > thr:
                worst_long = max(worst_long, err)
            else:
                worst_short = max(worst_short, err)
        assert worst_long <= 1e-6, (t, worst_long)
        assert worst_short <= 2e-5, (t, worst_short)
        lam_prev, T_prev = lam32, T32
    assert mp.plan_info()["n_groups"] == 0
    mp.close()


def test_threshold_above_every_ray_is_the_ungrouped_fp32_path(m):
    w = make_workload("room_small")
    a = gpu_map(m, w, long_ray_f64=100000)
    a.infer(w.iters)
    b = gpu_map(m, w)
    b.set_plan(8, 256, 0)
    b.infer(w.iters)
    assert torch.equal(a.marginals(), b.marginals())
    a.close()
    b.close()


def test_marginals_against_oracle(m):
    w = make_workload("room_small")
    mp = gpu_map(m, w, long_ray_f64=8)
    mp.infer(w.iters)
    p = mp.marginals().cpu().numpy().astype(np.float64).ravel()
    mp.close()
    ref = oracle.infer(w)["p"]
    assert np.percentile(np.abs(p - ref), 99.9) <= 1e-4
    assert np.abs(p - ref).max() <= 1e-3


def test_option_errors(m):
    w = make_workload("room_small")
    for opt in ({"long_ray_f64": -1}, {"long_ray_f64": 8, "precision": m.PREC_F64},
                {"long_ray_f64": 8, "variants": 1}):
        with pytest.raises(m.MRFError):
            m.Map(w.grid, w.prior, m.Options(**opt))
