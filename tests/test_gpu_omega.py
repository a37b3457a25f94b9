"""mrf_accuracy: the paper's accuracy metric (Section "Evaluation Metric for Probabilistic Occupancy Maps")
against the oracle's, pixel by pixel, on the same marginals.

Both sides walk every ray with the same FP32 slab arithmetic, so entry and exit ranges agree bit for bit;
the classification is FP64 on both sides, where the library's exp / log1p may differ from the host's in
the last bit, which can flip a near-tie.  The bar: per-pixel agreement on all but 1 in 10^4 evaluated rays,
and the same set of evaluated pixels exactly.
"""
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


def inferred(m, w, **opt):
    mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p, **opt))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters)
    return mp


def agree(m, mp, w, frames):
    p = mp.marginals().cpu().numpy().astype(np.float64).ravel()
    tot_acc = tot_ev = 0
    for fr in frames:
        n_acc, n_ev, res = mp.accuracy(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut,
                                       per_pixel=True)
        res = res.cpu().numpy().ravel()
        ref = oracle.omega_frame(w.grid, fr.cam, w.lut, fr.depth, p)
        assert np.array_equal(res >= 0, ref >= 0)
        ev = ref >= 0
        mism = int((res[ev] != ref[ev]).sum())
        assert mism <= max(1, ev.sum() // 10000), (mism, ev.sum())
        assert n_ev == int(ev.sum()) and n_acc == int((res == 1).sum())
        tot_acc += n_acc
        tot_ev += n_ev
    return tot_acc, tot_ev


@pytest.mark.parametrize("name", ["plain_64x48", "room_small", "diff_small"])
def test_accuracy_matches_oracle(m, name):
    w = make_workload(name)
    mp = inferred(m, w)
    frames = list(w.frames) + list(getattr(w, "heldout", []) or [])
    n_acc, n_ev = agree(m, mp, w, frames)
    assert n_ev > 0 and 0 < n_acc <= n_ev
    mp.close()


def test_accuracy_f64_map_and_counts_only(m):
    w = make_workload("room_small")
    mp = inferred(m, w, precision=m.PREC_F64)
    agree(m, mp, w, w.frames[:2])
    fr = w.frames[0]
    a = mp.accuracy(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    b = mp.accuracy(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut, per_pixel=True)
    assert a == b[:2]
    mp.close()


def test_accuracy_tracks_inference(m):
    """Inference raises the accuracy of the prior-only map on the frames it fused."""
    w = make_workload("room_small")
    mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    fr = w.frames[0]
    d = torch.from_numpy(fr.depth).cuda()
    mp.infer(0)
    a0, n0 = mp.accuracy(d, fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters)
    a1, n1 = mp.accuracy(d, fr.cam.pose, fr.cam, w.lut)
    assert n0 == n1 and a1 > a0
    mp.close()


def test_accuracy_errors(m):
    w = make_workload("room_small")
    fr = w.frames[0]
    mp = m.Map(w.grid, w.prior)
    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    with pytest.raises(m.MRFError, match="infer"):
        mp.accuracy(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.close()
    mp = m.Map([w.grid, w.grid], w.prior)
    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(1)
    with pytest.raises(m.MRFError, match="single-scene"):
        mp.accuracy(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.close()
