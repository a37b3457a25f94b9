"""The paper implementation's variants on the GPU (traversed-length weighting, per-keyframe average
messages) against the oracle's (tests/test_oracle_variants.py pins those).

First pass: every stored per-edge value (w lambda, averaged per (keyframe, voxel)) against the oracle's,
edge by edge.  Whole BP: the marginals, at the FP32 bar of the other whole-BP parity tests (parity_bars.py).
"""
import numpy as np
import pytest

import oracle
from synth import make_workload

from parity_bars import check_marginals, sensitivity_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("length", 1), ("keyframe", 2), ("both", 3)]


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as m
    m.build()
    return m


def gpu_map(m, w, variants, **opt):
    mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p, variants=variants, **opt))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    return mp


def oracle_variants(w, variants, iters):
    return oracle.infer_variants(w, length_weight=bool(variants & 1), keyframe_avg=bool(variants & 2),
                                 iters=iters)


def variant_sensitivity(w, variants, p_ref):
    """The variant oracle's own sensitivity to rounding-size noise on its likelihoods (parity_bars.py)."""
    csr = oracle.trace_frames(w.grid, w.frames, w.lut)
    ln = oracle.log_nu_edges(w.lut, csr["ray_off"], csr["Z"], csr["d"])
    wl = oracle.length_weights(w.grid, w.frames, w.lut) if variants & 1 else None
    rf = None
    if variants & 2:
        rf = np.concatenate([np.full(fr.cam.W * fr.cam.H, k, np.int32) for k, fr in enumerate(w.frames)])
    return sensitivity_map(csr["ray_off"], csr["vox"], ln, w.grid.n_voxels, w.prior, w.init_p or w.prior,
                           oracle.default_log_nu_bg(w.lut), w.iters, p_ref, bp=oracle.bp_variants, extra=(wl, rf))


@pytest.mark.parametrize("name", ["room_small", "diff_small"])
@pytest.mark.parametrize("case,variants", CASES)
def test_first_passes_edge_by_edge(m, name, case, variants):
    w = make_workload(name)
    mp = gpu_map(m, w, variants)
    for iters in (1, 2):
        mp.infer(iters)
        lam, _ = mp.export_messages()
        got = lam.double().cpu().numpy()
        ref = oracle_variants(w, variants, iters)["lam"]
        assert got.shape == ref.shape
        err = np.abs(got - ref) / (1 + np.abs(ref))
        # pass 2 starts from FP32 beliefs: allow the FP32 bar of one pass on top of the first pass's
        assert err.max() <= (2e-5 if iters == 1 else 1e-4), (iters, err.max())
    mp.close()


@pytest.mark.parametrize("name", ["plain_64x48", "room_small", "diff_small"])
@pytest.mark.parametrize("case,variants", CASES)
def test_marginals_match_oracle(m, name, case, variants):
    w = make_workload(name)
    mp = gpu_map(m, w, variants)
    mp.infer(w.iters)
    p = mp.marginals().cpu().numpy().astype(np.float64).ravel()
    if variants & 1:
        assert mp.plan_info()["n_groups"] == 0   # the tile-per-CTA kernel
    mp.close()
    ref = oracle_variants(w, variants, w.iters)["p"]
    exact = oracle.infer(w, init_p=w.init_p or w.prior)["p"]
    assert np.abs(ref - exact).max() > 1e-3          # the variant changes the answer
    check_marginals(p, ref, variant_sensitivity(w, variants, ref), f"{name} {case}")


def test_keyframe_average_in_a_batch_and_graph(m):
    """Batched contexts: pairs are per scene's frame; graph replay repeats the variant bitwise."""
    from synth.scenes import make_batch_small
    ws = make_batch_small()
    mp = m.Map([w.grid for w in ws], ws[0].prior, m.Options(variants=3))
    for s, w in enumerate(ws):
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut, scene=s)
    mp.infer(ws[0].iters)
    p = mp.marginals().clone()
    mp.infer_graph(ws[0].iters)
    assert torch.equal(p, mp.marginals())
    for s, w in enumerate(ws):
        ref = oracle_variants(w, 3, w.iters)["p"]
        ps = mp.scene_marginals(p, s).cpu().numpy().astype(np.float64).ravel()
        check_marginals(ps, ref, variant_sensitivity(w, 3, ref), f"scene {s}")
    mp.close()


def test_variant_errors(m):
    w = make_workload("diff_small")
    with pytest.raises(m.MRFError):
        m.Map(w.grid, w.prior, m.Options(precision=m.PREC_F64, variants=1))
    with pytest.raises(m.MRFError):
        m.Map(w.grid, w.prior, m.Options(variants=4))
    mp = gpu_map(m, w, 2)
    for fr in w.heldout:
        mp.add_heldout(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    with pytest.raises(m.MRFError, match="exact BP"):
        mp.grad(2, w.lut)
    mp.close()
