"""Pins for the FP64 oracle: checks against what the paper and mathematics fix.

None of these tests re-types the oracle's formulas.  The references are
literal enumerations of the definitions (oracle.brute), exact rational
fixtures, closed forms derived by hand from Eqs. "pos"/"neg", and geometric
brute force for the traversal.
"""
import math
from fractions import Fraction as F
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import make_workload
from synth.scenes import Camera, Grid, NoiseTable, look_at, noise_table

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ray_messages_exact.txt")


def logit(p):
    return np.log(p) - np.log1p(-p)


# --------------------------------------------------------------------------
# ray messages (Eqs. pos / neg) against enumeration of Eq. factor_to_node
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 9, 12, 14])
@pytest.mark.parametrize("nu_bg", [0.0, 0.02, 1.7])
def test_ray_messages_match_enumeration(N, nu_bg):
    rng = np.random.default_rng(100 * N + int(nu_bg * 10))
    for trial in range(3):
        m1 = rng.uniform(0.001, 0.999, N)
        if trial == 2:  # saturated incoming messages
            m1 = np.where(rng.random(N) < 0.5, 1e-6, 1 - 1e-6)
        nu = np.exp(rng.uniform(-6, 5, N))
        L = logit(m1)
        lbg = math.log(nu_bg) if nu_bg > 0 else -math.inf
        got = oracle.ray_messages(L, np.log(nu), lbg)
        with np.errstate(divide="ignore"):
            ref = np.clip(brute.factor_to_node(m1, nu, nu_bg), -64, 64)
        assert np.abs(got - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
        got2 = oracle.ray_messages_divfree(L, np.log(nu), lbg)
        assert np.abs(got2 - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def _read_golden():
    cases, trees = [], []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = [p.strip() for p in line.split("|")]
        if parts[0] == "TREE":
            prior = F(parts[1])
            nu = [F(x) for x in parts[2].split()]
            bg = F(parts[3])
            ps = [F(x) for x in parts[4].split()]
            trees.append((prior, nu, bg, ps))
        else:
            m1 = [F(x) for x in parts[1].split()]
            nu = [F(x) for x in parts[2].split()]
            bg = F(parts[3])
            mus = [tuple(F(y) for y in x.split(",")) for x in parts[4].split(";")]
            cases.append((m1, nu, bg, mus))
    return cases, trees


def test_ray_messages_exact_golden():
    cases, _ = _read_golden()
    assert len(cases) >= 5
    for m1, nu, bg, mus in cases:
        L = [math.log(float(x)) - math.log(float(1 - x)) for x in m1]
        lbg = math.log(float(bg)) if bg > 0 else -math.inf
        got = oracle.ray_messages(L, [math.log(float(x)) for x in nu], lbg)
        ref = [math.log(float(a)) - math.log(float(b)) for a, b in mus]
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_hand_worked_two_voxel_ray():
    """N = 2, mu(o=1) = (1/2, 1/3), nu = (2, 1), nu_bg = 1/2, worked by hand from Eqs. pos/neg.

    pos_1 = nu_1 P_1 = 2;  neg_1 = (w_2 + nu_bg P_3) / mu(o_1=0) = (1/6 + 1/6) * 2 = 2/3
    pos_2 = w_1 + nu_2 P_2 = 1 + 1/2 = 3/2;  neg_2 = w_1 + nu_bg P_3 / mu(o_2=0) = 1 + 1/4 = 5/4
    """
    got = oracle.ray_messages([0.0, math.log(0.5)], [math.log(2.0), 0.0], math.log(0.5))
    np.testing.assert_allclose(got, [math.log(3.0), math.log(6.0 / 5.0)], atol=1e-14)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
def test_uninformative_measurement_gives_zero_messages():
    """nu constant = c and nu_bg = c: pos_i = neg_i = c by telescoping, so lambda = 0."""
    rng = np.random.default_rng(3)
    for N in [1, 5, 40, 300]:
        c = float(rng.uniform(0.1, 10))
        L = rng.normal(0, 4, N)
        got = oracle.ray_messages(L, np.full(N, math.log(c)), math.log(c))
        assert np.abs(got).max() < 1e-11


def test_constant_nu_without_background():
    """nu constant and nu_bg = 0: lambda_i = -log(1 - P_{N+1} / mu(o_i = 0))."""
    rng = np.random.default_rng(4)
    for N in [2, 7, 30]:
        m1 = rng.uniform(0.05, 0.95, N)
        m0 = 1 - m1
        PN1 = np.prod(m0)
        ref = -np.log(1 - PN1 / m0)
        got = oracle.ray_messages(logit(m1), np.full(N, 0.3), -math.inf)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


def test_single_voxel_ray():
    """N = 1: pos = nu_1, neg = nu_bg, so lambda = log(nu_1 / nu_bg), whatever mu(o_1)."""
    for L in [-5.0, 0.0, 3.0]:
        got = oracle.ray_messages([L], [math.log(2.5)], math.log(0.1))
        assert abs(got[0] - math.log(25.0)) < 1e-13
    got = oracle.ray_messages([0.0], [0.0], -math.inf)
    assert got[0] == 64.0  # infinite message clamped


def test_message_does_not_depend_on_own_incoming():
    """A factor->node message excludes the node's own incoming message (Eq. factor_to_node)."""
    rng = np.random.default_rng(5)
    L = rng.normal(0, 2, 8)
    ln = rng.normal(0, 1, 8)
    a = oracle.ray_messages(L, ln, -1.0)
    for i in range(8):
        L2 = L.copy()
        L2[i] += 7.0
        b = oracle.ray_messages(L2, ln, -1.0)
        assert abs(a[i] - b[i]) < 1e-12
        assert np.abs(np.delete(a - b, i)).max() > 1e-6


# --------------------------------------------------------------------------
# inference: trees are exact, loopy graphs match generic sum-product
# --------------------------------------------------------------------------
def test_tree_marginals_exact_golden():
    _, trees = _read_golden()
    for prior, nu, bg, ps in trees:
        N = len(nu)
        for iters in [1, 2, 4]:
            lam, T, p = oracle.bp(np.array([0, N]), np.arange(N, dtype=np.uint32),
                                  np.log([float(x) for x in nu]), N, float(prior), float(prior),
                                  math.log(float(bg)), iters)
            np.testing.assert_allclose(p, [float(x) for x in ps], atol=1e-13)


@pytest.mark.parametrize("N", [1, 3, 8, 13])
def test_tree_marginals_random(N):
    rng = np.random.default_rng(N)
    prior = float(rng.uniform(0.05, 0.9))
    nu = np.exp(rng.uniform(-3, 4, N))
    bg = float(np.exp(rng.uniform(-4, 0)))
    ref = brute.tree_marginals(prior, nu, bg)
    for init_p, first_exact in [(prior, 1), (0.1, 2)]:
        lam, T, p = oracle.bp(np.array([0, N]), np.arange(N, dtype=np.uint32), np.log(nu), N,
                              prior, init_p, math.log(bg), first_exact)
        np.testing.assert_allclose(p, ref, atol=1e-11)
        lam, T, p = oracle.bp(np.array([0, N]), np.arange(N, dtype=np.uint32), np.log(nu), N,
                              prior, init_p, math.log(bg), first_exact + 3)
        np.testing.assert_allclose(p, ref, atol=1e-11)


def _random_graph(rng, n_rays, V):
    rays = [list(rng.permutation(V)[: int(rng.integers(2, min(V, 7) + 1))]) for _ in range(n_rays)]
    nus = [np.exp(rng.uniform(-2, 3, len(r))) for r in rays]
    return rays, nus


@pytest.mark.parametrize("seed", range(6))
def test_loopy_bp_matches_generic_sum_product(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(4, 12))
    rays, nus = _random_graph(rng, int(rng.integers(2, 7)), V)
    prior = float(rng.uniform(0.1, 0.7))
    bg = [0.05, 0.5, 0.0][seed % 3]
    ro = np.cumsum([0] + [len(r) for r in rays])
    vox = np.concatenate(rays).astype(np.uint32)
    ln = np.log(np.concatenate(nus))
    for init_p in [prior, 0.1]:
        for iters in [0, 1, 2, 3, 6]:
            ref = brute.loopy_bp(rays, nus, bg, V, prior, init_p, iters)
            _, _, p = oracle.bp(ro, vox, ln, V, prior, init_p, math.log(bg) if bg > 0 else -math.inf, iters)
            np.testing.assert_allclose(p, ref, atol=1e-10)


def test_untouched_voxels_keep_prior_and_iters0():
    w = make_workload("plain_64x48")
    r0 = oracle.infer(w, iters=0)
    assert np.all(r0["p"] == pytest.approx(w.prior, abs=1e-15))
    r = oracle.infer(w)
    p = r["p"]
    assert np.all((p >= 0) & (p <= 1))
    touched = np.zeros(w.grid.n_voxels, bool)
    touched[r["csr"]["vox"]] = True
    assert np.abs(p[~touched] - w.prior).max() < 1e-15
    assert np.abs(p[touched] - w.prior).max() > 0.4
    r2 = oracle.infer(w)
    assert np.array_equal(r2["p"], p)


# --------------------------------------------------------------------------
# transpose
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(3))
def test_transpose_is_the_stable_sort_by_voxel(seed):
    """Each voxel's edge list is its edges in increasing edge order: numpy's stable argsort by voxel, and
    the offsets are the running counts (empty voxels included)."""
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 60))
    vox = rng.integers(0, V, int(rng.integers(0, 500))).astype(np.uint32)
    vstart, eid = oracle.transpose(vox, V)
    np.testing.assert_array_equal(eid, np.argsort(vox, kind="stable"))
    np.testing.assert_array_equal(vstart, np.r_[0, np.cumsum(np.bincount(vox, minlength=V))])


# --------------------------------------------------------------------------
# sensor likelihood
# --------------------------------------------------------------------------
def test_log_nu_is_a_normalised_density_in_Z():
    lut = noise_table(64, 8.87)
    lut.outlier_w = 0.02
    for d in [0.7, 2.0, 4.5]:
        zz = np.linspace(d - 0.5, d + 0.5, 4001)
        g = np.exp(np.array([oracle.log_nu(lut, d, z) for z in zz]))
        # the Gaussian part integrates to (1-w); the floor adds w/d_hi per metre of Z
        integral = np.trapezoid(g, zz) - lut.outlier_w / lut.d_hi * 1.0
        assert abs(integral - (1 - lut.outlier_w)) < 1e-6
        zz = zz[::4]
        peak = max(zz, key=lambda z: oracle.log_nu(lut, d, z))
        assert abs(peak - d) < 1e-3


def test_edge_likelihoods_and_background():
    """The per-edge evaluation is the pointwise one, edge by edge with its ray's Z; the all-empty
    likelihood is the outlier floor w / d_hi."""
    lut = noise_table(64, 8.87)
    rng = np.random.default_rng(3)
    ray_off = np.array([0, 3, 3, 7, 12], np.int64)                 # an empty ray included
    Z = rng.uniform(0.5, 6.0, 4).astype(np.float32)
    d = rng.uniform(0.3, 7.0, 12).astype(np.float32)
    ln = oracle.log_nu_edges(lut, ray_off, Z, d)
    for r in range(4):
        for e in range(ray_off[r], ray_off[r + 1]):
            assert ln[e] == pytest.approx(oracle.log_nu(lut, float(d[e]), float(Z[r])), abs=1e-12)
    assert oracle.default_log_nu_bg(lut) == pytest.approx(math.log(float(np.float32(lut.outlier_w))
                                                                    / float(np.float32(lut.d_hi))), abs=1e-12)


def test_log_sigma_table_interpolation():
    lut = NoiseTable(8, 0.0, 4.0, np.log(np.linspace(0.01, 0.08, 8)).astype(np.float32), 0.0)
    delta = 0.5
    for k in range(8):
        c = (k + 0.5) * delta
        assert oracle.log_sigma_at(lut, c) == pytest.approx(float(lut.log_sigma[k]), abs=1e-15)
    mid = oracle.log_sigma_at(lut, 2 * delta)  # halfway between centres 1 and 2... of bins 1,2
    assert mid == pytest.approx(0.5 * (float(lut.log_sigma[1]) + float(lut.log_sigma[2])), abs=1e-12)
    assert oracle.log_sigma_at(lut, -3.0) == pytest.approx(float(lut.log_sigma[0]), abs=1e-15)
    assert oracle.log_sigma_at(lut, 99.0) == pytest.approx(float(lut.log_sigma[7]), abs=1e-15)
    # Gaussian value at the mean: log nu = -log sigma - log sqrt(2 pi) when w = 0
    assert oracle.log_nu(lut, 0.25, 0.25) == pytest.approx(-float(lut.log_sigma[0]) - 0.5 * math.log(2 * math.pi))


def test_bias_table_shifts_the_predicted_measurement():
    """Section IV-C: the bias predicts the mean measurement, d + b(d); the density is the unbiased one moved
    by b (closed form: the peak value and the whole profile in Z), with b interpolated like log sigma."""
    base = noise_table(32, 8.0)
    base.outlier_w = 0.0
    bias = np.linspace(-0.02, 0.03, 32).astype(np.float32)
    lut = NoiseTable(base.n_bins, base.d_lo, base.d_hi, base.log_sigma, 0.0, bias)
    delta = (base.d_hi - base.d_lo) / base.n_bins
    for k in [0, 7, 20, 31]:
        d = base.d_lo + (k + 0.5) * delta       # a bin centre: b(d) is the table entry
        b = float(bias[k])
        for dz in [-0.01, 0.0, 0.004]:
            assert oracle.log_nu(lut, d, d + b + dz) == pytest.approx(oracle.log_nu(base, d, d + dz), abs=1e-12)
    # between two centres the bias is the linear blend
    d = base.d_lo + 10.75 * delta
    b = 0.75 * float(bias[10]) + 0.25 * float(bias[11])
    assert oracle.log_nu(lut, d, d + b) == pytest.approx(oracle.log_nu(base, d, d), abs=1e-12)


# --------------------------------------------------------------------------
# traversal against geometric brute force
# --------------------------------------------------------------------------
def _tiny_cases(seed, n_cams=6):
    rng = np.random.default_rng(seed)
    out = []
    for ci in range(n_cams):
        n = int(rng.integers(5, 17))
        grid = Grid(n, int(rng.integers(5, 17)), int(rng.integers(5, 17)), float(rng.uniform(0.05, 0.2)),
                    tuple(rng.uniform(-0.3, 0.3, 3)))
        ext = grid.extent
        centre = np.array(grid.origin) + ext / 2
        inside = ci % 2 == 0
        if inside:
            c = np.array(grid.origin) + rng.uniform(0.1, 0.9, 3) * ext
        else:
            c = centre + rng.normal(0, 1, 3) / 1 * np.linalg.norm(ext)
        target = centre + rng.normal(0, 0.2, 3) * ext
        W, H = 12, 9
        cam = Camera(W, H, 9.0, 9.0, 5.5, 4.0, look_at(c, target))
        depth = rng.uniform(0.05, 2 * np.linalg.norm(ext), (H, W)).astype(np.float32)
        depth[rng.random((H, W)) < 0.1] = 0.0
        lut = noise_table(16, grid.diagonal)
        out.append((grid, cam, depth, lut))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_traversal_matches_fine_marching_and_slabs(seed):
    mism = 0
    total = 0
    for grid, cam, depth, lut in _tiny_cases(seed):
        tr = oracle.trace_frame(grid, cam, depth, lut)
        n = (grid.nx, grid.ny, grid.nz)
        rays = tr["rays"]
        for r in range(len(rays)):
            ry = rays[r]
            N = int(ry["N"])
            vox = tr["vox"][tr["ray_off"][r]:tr["ray_off"][r + 1]]
            d = tr["d"][tr["ray_off"][r]:tr["ray_off"][r + 1]]
            if N == 0:
                continue
            total += 1
            cells = [(int(v % n[0]), int((v // n[0]) % n[1]), int(v // (n[0] * n[1]))) for v in vox]
            assert len(set(cells)) == N
            # consecutive cells are face neighbours, ending at the closed-form end voxel
            for a, b in zip(cells[:-1], cells[1:]):
                assert sum(abs(x - y) for x, y in zip(a, b)) == 1
            assert cells[0] == tuple(int(x) for x in ry["s"]) and cells[-1] == tuple(int(x) for x in ry["e"])
            # depths are segment midpoints: non-decreasing and inside [t0, t1]
            assert np.all(np.diff(d) >= 0) and d[0] >= ry["t0"] and d[-1] <= ry["t1"]
            o, k = ry["o"].astype(np.float64), ry["k"].astype(np.float64)
            t0, t1 = float(ry["t0"]), float(ry["t1"])
            seg = brute.segment_lengths(o, k, t0, t1, n)
            for c, ln in seg.items():   # every voxel the segment really crosses is visited
                if ln > 1e-4:
                    assert c in set(cells), (c, ln)
            for c in cells:             # every visited voxel touches the segment
                assert seg.get(c, -1.0) >= -1e-6 or c in seg, c
            march = brute.march_cells(o, k, t0, t1, n, step=2e-5)
            if march != cells:
                mism += 1
                disputed = set(march) ^ set(cells)
                assert all(seg.get(c, 0.0) < 1e-4 for c in disputed), disputed
    assert total > 100
    assert mism <= max(2, total // 50)


def test_truncation_three_sigma():
    """Rays stop 3 sigma beyond the measured range (Section IV-B) or at the grid exit."""
    w = make_workload("plain_64x48")
    fr = w.frames[0]
    rays = oracle.frame_setup(w.grid, fr.cam, fr.depth, w.lut)
    v = rays["N"] > 0
    Z = rays["Z"][v].astype(np.float64)
    t1 = rays["t1"][v].astype(np.float64)
    sig = np.exp([oracle.log_sigma_at(w.lut, z) for z in Z])
    assert np.all(t1 <= Z + 3 * sig * 1.05 + 1e-5)
    inner = t1 < Z + 3 * sig * 0.95
    # rays cut short are the ones leaving the grid: their end point is on the grid boundary
    for r in np.nonzero(v)[0][inner]:
        p = rays["o"][r].astype(np.float64) + float(rays["t1"][r]) * rays["k"][r].astype(np.float64)
        n = np.array([w.grid.nx, w.grid.ny, w.grid.nz])
        assert np.min(np.minimum(np.abs(p), np.abs(p - n))) < 1e-3
