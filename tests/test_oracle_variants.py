"""Pins of the oracle's implementation variants (Section "Belief Propagation" of the implementation):
traversed-length weighting and per-keyframe average messages.

Readings (stated in the oracle): a ray's log-odds message enters a voxel's belief as w lambda with
w = min(1, l / h), l the traversed length; the cavity leaves out the ray's own w lambda; with averaging,
all rays of one keyframe through a voxel send the mean of their (weighted) messages, and the cavity
leaves out that mean.

What fixes them, independently of the oracle's code:
  * a single ray is a tree: with weights its beliefs must be logit gamma + w_i lambda_i with lambda_i the
    exact tree message from brute-force enumeration (so its marginals are fixed in closed form);
  * averaging over groups of one message, or of identical messages, changes nothing: exact BP (itself
    pinned to brute force elsewhere) is the answer;
  * the weights come from the traversed lengths, which exact slab clipping fixes.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import make_workload


def random_graph(rng, R=12, V=30, nmax=9):
    offs, vox, ln = [0], [], []
    for _ in range(R):
        n = int(rng.integers(1, nmax + 1))
        vox += list(rng.choice(V, n, replace=False))
        ln += list(rng.normal(0.0, 2.0, n))
        offs.append(len(vox))
    return np.array(offs, np.int64), np.array(vox, np.uint32), np.array(ln)


LBG = math.log(0.05)


@pytest.mark.parametrize("iters", [1, 3, 7])
def test_variants_off_and_trivial_are_exact_bp(iters):
    rng = np.random.default_rng(iters)
    ro, vx, ln = random_graph(rng)
    R, E = len(ro) - 1, int(ro[-1])
    _, T0, p0 = oracle.bp(ro, vx, ln, 30, 0.3, 0.1, LBG, iters)
    for wl, rf in [(None, None), (np.ones(E), None), (None, np.arange(R)), (np.ones(E), np.arange(R))]:
        _, T, p = oracle.bp_variants(ro, vx, ln, 30, 0.3, 0.1, LBG, iters, wl, rf)
        assert np.array_equal(T, T0) and np.array_equal(p, p0)
    # one frame for every ray does change a loopy graph: the averaging is live
    _, _, p1 = oracle.bp_variants(ro, vx, ln, 30, 0.3, 0.1, LBG, iters, None, np.zeros(R))
    if iters > 1:
        assert np.abs(p1 - p0).max() > 1e-3


def test_average_of_identical_rays_is_exact():
    """Two copies of each ray in one frame receive identical messages, so their average is exact and the
    belief must count both copies."""
    rng = np.random.default_rng(5)
    ro, vx, ln = random_graph(rng, R=6, V=14)
    offs, vv, ll, frame = [0], [], [], []
    for r in range(len(ro) - 1):
        a, b = ro[r], ro[r + 1]
        for _ in range(2):
            vv += list(vx[a:b])
            ll += list(ln[a:b])
            offs.append(len(vv))
            frame.append(r)
    ro2, vx2, ln2 = np.array(offs), np.array(vv, np.uint32), np.array(ll)
    _, T0, p0 = oracle.bp(ro2, vx2, ln2, 14, 0.4, 0.1, LBG, 6)
    _, T1, p1 = oracle.bp_variants(ro2, vx2, ln2, 14, 0.4, 0.1, LBG, 6, None, np.array(frame))
    np.testing.assert_allclose(T1, T0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_length_weights_on_a_single_ray(seed):
    """A tree: every message is the exact one, and the belief of voxel i is logit gamma + w_i lambda_i."""
    rng = np.random.default_rng(seed)
    N = int(rng.integers(2, 11))
    nu = np.exp(rng.normal(0.0, 1.5, N))
    nu_bg, prior = 0.2, 0.35
    w = rng.uniform(0.05, 1.0, N)
    exact = brute.tree_marginals(prior, nu, nu_bg)
    lg = math.log(prior / (1 - prior))
    lam = np.log(exact / (1 - exact)) - lg
    want = 1.0 / (1.0 + np.exp(-(lg + w * lam)))
    ro = np.array([0, N])
    for iters, init in [(1, prior), (2, 0.1), (5, 0.1)]:
        _, T, p = oracle.bp_variants(ro, np.arange(N, dtype=np.uint32), np.log(nu), N, prior, init,
                                     math.log(nu_bg), iters, w, None)
        np.testing.assert_allclose(T, lg + w * lam, rtol=0, atol=1e-10)
        np.testing.assert_allclose(p, want, rtol=0, atol=1e-12)
        # with averaging on top (one ray: groups of one) nothing changes
        _, T2, _ = oracle.bp_variants(ro, np.arange(N, dtype=np.uint32), np.log(nu), N, prior, init,
                                      math.log(nu_bg), iters, w, np.zeros(1))
        assert np.array_equal(T2, T)


def test_length_weights_against_slab_clipping():
    w = make_workload("room_small")
    g = w.grid
    fr = w.frames[0]
    wl = oracle.length_weights(g, [fr], w.lut)
    rays = oracle.frame_setup(g, fr.cam, fr.depth, w.lut)
    off = np.zeros(len(rays) + 1, np.int64)
    np.cumsum(rays["N"].astype(np.int64), out=off[1:])
    assert len(wl) == off[-1] and wl.min() >= 0 and wl.max() <= 1
    rng = np.random.default_rng(1)
    checked = 0
    for r in rng.permutation(len(rays)):
        if rays["N"][r] == 0:
            continue
        ry = rays[r]
        lens = brute.segment_lengths(ry["o"], ry["k"], float(ry["t0"]), float(ry["t1"]), (g.nx, g.ny, g.nz))
        ref = np.sort([min(1.0, x) for x in lens.values() if x > 1e-9])
        got = np.sort(wl[off[r]:off[r + 1]][wl[off[r]:off[r + 1]] > 1e-6])
        if len(ref) != len(got):   # a corner touched within rounding: the FP32 walk may list it
            continue
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)
        checked += 1
        if checked == 200:
            break
    assert checked == 200
