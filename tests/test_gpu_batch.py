"""Batched contexts (many scenes as one), caller-chosen kernel plans and CUDA-graph replay."""
import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.scenes import make_batch_small

from parity_bars import check_marginals, workload_sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_TOL = 1e-4


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as m
    m.build()
    return m


def single(m, w, iters=None):
    mp = m.Map(w.grid, w.prior)
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters if iters is None else iters)
    return mp


def batched(m, ws):
    mp = m.Map([w.grid for w in ws], ws[0].prior)
    for s, w in enumerate(ws):
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut, scene=s)
    return mp


def test_batch_matches_each_scene_alone_and_the_oracle(m):
    ws = make_batch_small()
    assert len({w.iters for w in ws}) == 1
    mp = batched(m, ws)
    mp.infer(ws[0].iters)
    p = mp.marginals()
    assert mp.n_voxels == sum(w.grid.n_voxels for w in ws)
    for s, w in enumerate(ws):
        ps = mp.scene_marginals(p, s).cpu().numpy().astype(np.float64).ravel()
        one = single(m, w)
        p1 = one.marginals().cpu().numpy().astype(np.float64).ravel()
        one.close()
        # the same arithmetic; only rounding orders can differ (the other scenes' edges move the tile
        # boundaries, so the CTA scans and the per-tile partial sums group differently), which BP may
        # amplify: the FP32 bar
        assert np.max(np.abs(ps - p1)) <= P_TOL, (s, np.max(np.abs(ps - p1)))
        ref = oracle.infer(w)
        check_marginals(ps, ref["p"], workload_sensitivity(w, ref), f"scene {s}")
    mp.close()


def test_batch_scenes_are_independent(m):
    """A scene's marginals do not depend on the other scenes' frames."""
    import dataclasses
    ws = make_batch_small()
    a = batched(m, ws)
    a.infer(ws[0].iters)
    pa = a.scene_marginals(a.marginals(), 1).clone()
    a.close()
    fewer = dataclasses.replace(ws[0], frames=ws[0].frames[:1])
    b = batched(m, [fewer, ws[1], ws[2]])
    b.infer(ws[0].iters)
    # the other scene's edges move scene 1's tile boundaries, so only rounding may differ
    assert torch.allclose(pa, b.scene_marginals(b.marginals(), 1), atol=1e-5)
    b.close()


def test_batch_errors(m):
    ws = make_batch_small()
    mp = batched(m, ws)
    fr = ws[0].frames[0]
    with pytest.raises(m.MRFError):
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, ws[0].lut, scene=7)
    mp.infer(2)
    with pytest.raises(m.MRFError, match="single-scene"):
        mp.export_rays()
    with pytest.raises(m.MRFError, match="single-scene"):
        mp.add_heldout(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, ws[0].lut)
    mp.close()


def test_infer_graph_replays_infer_bitwise(m):
    w = make_workload("room_small")
    mp = single(m, w)
    p_ref = mp.marginals().clone()
    for _ in range(3):   # record, then replay twice
        mp.infer_graph(w.iters)
        assert torch.equal(mp.marginals(), p_ref)
    mp.infer_graph(3)    # another iters value records again
    mp.infer(3)
    p3 = mp.marginals().clone()
    mp.infer_graph(3)
    assert torch.equal(mp.marginals(), p3)
    # new frames drop the recording
    fr = w.frames[0]
    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters)
    p_new = mp.marginals().clone()
    assert not torch.equal(p_new, p_ref)
    mp.infer_graph(w.iters)
    assert torch.equal(mp.marginals(), p_new)
    mp.close()


def test_infer_graph_on_a_batch(m):
    ws = make_batch_small()
    mp = batched(m, ws)
    mp.infer(ws[0].iters)
    p_ref = mp.marginals().clone()
    mp.infer_graph(ws[0].iters)
    mp.infer_graph(ws[0].iters)
    assert torch.equal(mp.marginals(), p_ref)
    mp.close()


_SENS = {}


def _room_small_sensitivity(w, ref):
    """The oracle's sensitivity on the 4-frame room, computed once for the plan cases."""
    if "room_small" not in _SENS:
        _SENS["room_small"] = workload_sensitivity(w, ref)
    return _SENS["room_small"]


@pytest.mark.parametrize("plan,expect", [
    ((8, 256, 1), (8, True)), ((8, 256, 0), (8, False)), ((16, 128, 1), (16, True)),
    ((16, -1, 0), (16, False)), ((32, -1, 0), (32, False)), ((32, 256, 1), (32, False)),
    ((4, 512, 1), (4, True)), ((4, 512, 0), (4, False)),
])
def test_set_plan(m, plan, expect):
    w = make_workload("room_small")
    mp = m.Map(w.grid, w.prior)
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.set_plan(*plan)
    mp.infer(w.iters)
    info = mp.plan_info()
    assert info["ray_items"] == expect[0] and (info["n_groups"] > 0) == expect[1]
    p = mp.marginals().cpu().numpy().astype(np.float64).ravel()
    ref = oracle.infer(w)
    check_marginals(p, ref["p"], _room_small_sensitivity(w, ref), f"plan {plan}")
    with pytest.raises(m.MRFError):
        mp.set_plan(12, 0, -1)
    mp.close()
