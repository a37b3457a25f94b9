"""mrf_grad: gradient of the held-out depth likelihood with respect to the noise table.

Compared with the FP64 oracle's adjoint (tests/test_oracle_grad.py pins it to
central differences) and directly with central differences of the oracle's
loss, at a table 30% off the generating one (where a fit would start).  The
bar is 1e-3 relative, in norm and per component (plus 1e-4 of the largest
component for the near-zero ones).
"""
import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.scenes import NoiseTable, theta_off

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as m
    m.build()
    return m


def make_map(m, w, theta, **opt):
    mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p, **opt))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, theta)
    for fr in w.heldout:
        mp.add_heldout(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, theta)
    return mp


def oracle_problem(w, theta):
    return (oracle.trace_frames(w.grid, w.frames, theta), oracle.trace_frames(w.grid, w.heldout, theta))


def close(g, ref, rel=1e-3):
    g, ref = np.asarray(g), np.asarray(ref)
    assert np.linalg.norm(g - ref) <= rel * np.linalg.norm(ref), (np.linalg.norm(g - ref), np.linalg.norm(ref))
    assert np.all(np.abs(g - ref) <= rel * np.abs(ref) + 1e-4 * np.abs(ref).max()), np.c_[g, ref]


@pytest.mark.parametrize("iters", [0, 1, 6])
def test_grad_matches_oracle_adjoint(m, iters):
    w = make_workload("diff_small")
    th = theta_off(w.lut)
    mp = make_map(m, w, th)
    loss, g_ls, g_w = mp.grad(iters, th)
    mp.close()
    tr, ho = oracle_problem(w, th)
    lo, gls_o, gw_o = oracle.grad(th, th.log_sigma.astype(np.float64), float(th.outlier_w), tr, ho,
                                  w.grid.n_voxels, w.prior, w.init_p, iters)
    assert loss == pytest.approx(lo, rel=1e-5)
    close(np.r_[g_ls, g_w], np.r_[gls_o, gw_o])


@pytest.mark.parametrize("table", ["bias", "outlier_0.3"])
def test_grad_table_variants_match_oracle_adjoint(m, table):
    """A bias table (the likelihood's mean moved by b(d), up to 4 mm) and a large outlier
    weight: both move the far-edge distances past which the kernels take an edge's
    likelihood as the floor (the bias widens them; w sets the floor they are measured
    against)."""
    w = make_workload("diff_small")
    th = theta_off(w.lut)
    if table == "bias":
        k = np.arange(th.n_bins)
        th = NoiseTable(th.n_bins, th.d_lo, th.d_hi, th.log_sigma, th.outlier_w,
                        (0.004 * np.sin(0.7 * k)).astype(np.float32))
    else:
        th = NoiseTable(th.n_bins, th.d_lo, th.d_hi, th.log_sigma, 0.3, th.bias)
    mp = make_map(m, w, th)
    loss, g_ls, g_w = mp.grad(4, th)
    mp.close()
    tr, ho = oracle_problem(w, th)
    lo, gls_o, gw_o = oracle.grad(th, th.log_sigma.astype(np.float64), float(th.outlier_w), tr, ho,
                                  w.grid.n_voxels, w.prior, w.init_p, 4)
    assert loss == pytest.approx(lo, rel=1e-5)
    close(np.r_[g_ls, g_w], np.r_[gls_o, gw_o])


def test_grad_matches_central_differences(m):
    """The target bar: adjoint gradient within 1e-3 of central differences (h = 1e-6, FP64 oracle)."""
    w = make_workload("diff_small")
    th = theta_off(w.lut)
    mp = make_map(m, w, th)
    _, g_ls, g_w = mp.grad(w.iters, th)
    mp.close()
    tr, ho = oracle_problem(w, th)
    theta = np.r_[th.log_sigma.astype(np.float64), float(th.outlier_w)]

    def f(x):
        return oracle.grad(th, x[:-1], x[-1], tr, ho, w.grid.n_voxels, w.prior, w.init_p, w.iters, with_grad=False)

    h = 1e-6
    fd = np.array([(f(theta + h * e) - f(theta - h * e)) / (2 * h) for e in np.eye(len(theta))])
    close(np.r_[g_ls, g_w], fd)


def test_grad_bitwise_deterministic_and_leaves_the_map_inferred(m):
    w = make_workload("diff_small")
    th = theta_off(w.lut)
    mp = make_map(m, w, th)
    a = mp.grad(w.iters, th)
    p1 = mp.marginals().clone()
    b = mp.grad(w.iters, th)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]
    mp.infer(w.iters)
    assert torch.equal(p1, mp.marginals())
    mp.close()


def test_grad_through_torch_autograd(m):
    w = make_workload("diff_small")
    th = theta_off(w.lut)
    mp = make_map(m, w, th)
    ls = torch.tensor(th.log_sigma.astype(np.float64), requires_grad=True)
    ow = torch.tensor(float(th.outlier_w), dtype=torch.float64, requires_grad=True)
    loss = m.HeldoutLoss.apply(ls, ow, mp, w.iters, th)
    (2.0 * loss).backward()
    _, g_ls, g_w = mp.grad(w.iters, th)
    assert np.allclose(ls.grad.numpy(), 2.0 * g_ls) and abs(float(ow.grad) - 2.0 * g_w) <= 1e-12 * abs(g_w)
    # a small step down the gradient lowers the loss
    with torch.no_grad():
        step = 1e-3 / float(ls.grad.abs().max())
        ls2 = ls - step * ls.grad
    loss2 = m.HeldoutLoss.apply(ls2, ow.detach(), mp, w.iters, th)
    assert float(loss2) < float(loss)
    mp.close()


def test_grad_errors(m):
    w = make_workload("diff_small")
    th = theta_off(w.lut)
    mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, th)
    with pytest.raises(m.MRFError, match="held-out"):
        mp.grad(w.iters, th)
    mp.close()
    mp = m.Map(w.grid, w.prior, m.Options(precision=m.PREC_F64))
    mp.add_frame(torch.from_numpy(w.frames[0].depth).cuda(), w.frames[0].cam.pose, w.frames[0].cam, th)
    mp.add_heldout(torch.from_numpy(w.heldout[0].depth).cuda(), w.heldout[0].cam.pose, w.heldout[0].cam, th)
    with pytest.raises(m.MRFError, match="FP32"):
        mp.grad(w.iters, th)
    mp.close()


def test_grad_full_workload_matches_golden(m):
    """8 + 2 frames of 160x120 over 128^3, 10 passes: against the oracle's central differences and adjoint
    stored by tests/golden/make_grad_golden.py."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "grad_diff_8x160x120.json")) as f:
        gold = json.load(f)
    w = make_workload("diff_8x160x120")
    th = theta_off(w.lut)
    mp = make_map(m, w, th)
    assert mp.stats()["n_edges"] == gold["edges"]
    loss, g_ls, g_w = mp.grad(gold["passes"], th)
    mp.close()
    assert loss == pytest.approx(gold["loss"], rel=1e-5)
    close(np.r_[g_ls, g_w], gold["grad_fd"])
    close(np.r_[g_ls, g_w], gold["grad_adjoint"])
