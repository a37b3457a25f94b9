"""The log-domain FP32 ablation (MRF_PREC_F32_LOG) against the FP64 oracle.

The ablation evaluates Eqs. "pos"/"neg" as the paper does, in the log domain
(log P by a Kahan-compensated prefix sum, log A and log B by log-add-exp
recurrences), in FP32.  It computes the same BP as the default path, so its
marginals follow the oracle's; how closely is what the ablation measures:
lambda = log pos - log neg cancels where pos and neg are close, so its error
grows with |log A| (long rays).  Measured on a GB300: max 7.1e-6 (64x48) and
3.9e-3 (4-frame room), p99.9 5.6e-7 and 2.3e-6, against 1.5e-6 and 2.3e-6 max
for the default FP32 form.  The bars are those figures with a margin of 2.5-4x.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import make_workload


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as mod
    mod.build()
    return mod


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["plain_64x48", "room_small"])
def test_log_domain_ablation_follows_the_oracle(m, name):
    w = make_workload(name)
    ref = oracle.infer(w)
    out = {}
    for prec in (m.PREC_F32, m.PREC_F32_LOG):
        mp = m.Map(w.grid, w.prior, m.Options(precision=prec, init_p=w.init_p))
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
        mp.infer(w.iters)
        out[prec] = np.abs(mp.marginals().double().cpu().numpy().ravel() - ref["p"])
        if prec == m.PREC_F32_LOG:
            assert mp.plan_info()["n_groups"] == 0   # thread-per-ray kernel, per-edge voxel totals
        mp.close()
    err_log, err_f32 = out[m.PREC_F32_LOG], out[m.PREC_F32]
    print(name, "log-domain FP32 max", err_log.max(), "p99.9", np.percentile(err_log, 99.9),
          "default FP32 max", err_f32.max())
    assert np.isfinite(err_log).all()
    assert err_log.max() <= 1e-2, err_log.max()
    assert np.percentile(err_log, 99.9) <= 1e-5
