"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every input is seeded and synthetic.  Bars (each derived from the FP32 arithmetic of the kernels):
  traversal (ray offsets, voxel ids, midpoint ranges, measured ranges): bit-exact
  transpose (perm, segments): exact
  FP32 marginals: |p - p_oracle| <= 1e-4 on every voxel where the oracle's own sensitivity to
    rounding-size noise is below 5e-6, else a bar scaled by it (parity_bars.py)
  FP64 marginals: |p - p_oracle| <= 1e-9
  ray messages on given inputs: |dlam| <= 2e-5 (1 + |lam|)
  voxel totals on given inputs: |dT| <= 1e-5 (1 + sum |lam|)
"""
import math

import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.scenes import Camera, Grid, look_at, noise_table

from parity_bars import check_marginals, workload_sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_TOL_F32 = 1e-4
P_TOL_F64 = 1e-9


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as mod
    mod.build()
    return mod


def run_map(m, w, frames=None, iters=None, **opt):
    frames = w.frames if frames is None else frames
    mp = m.Map(w.grid, w.prior, m.Options(**opt))
    for fr in frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters if iters is None else iters)
    return mp


# --------------------------------------------------------------------------
# traversal: bit-exact against the oracle's copy of the pinned recipe
# --------------------------------------------------------------------------
def _check_traversal(mp, ref):
    ex = mp.export_rays()
    np.testing.assert_array_equal(ex["ray_off"].cpu().numpy(), ref["ray_off"])
    np.testing.assert_array_equal(ex["vox"].cpu().numpy().view(np.uint32), ref["vox"])
    np.testing.assert_array_equal(ex["d"].cpu().numpy().view(np.uint32), ref["d"].view(np.uint32))
    np.testing.assert_array_equal(ex["Z"].cpu().numpy().view(np.uint32), ref["Z"].view(np.uint32))


@pytest.mark.parametrize("name", ["plain_64x48", "room_small"])
def test_traversal_bit_exact(m, name):
    w = make_workload(name)
    mp = run_map(m, w, iters=0)
    _check_traversal(mp, oracle.trace_frames(w.grid, w.frames, w.lut))
    mp.close()


@pytest.mark.parametrize("corner", [False, True])
def test_traversal_bit_exact_odd_cameras(m, corner):
    # corner: the camera on a voxel corner of a grid at the origin, looking along a
    # diagonal, so that face times of different axes coincide (the lower axis steps first)
    rng = np.random.default_rng(11 + corner)
    for trial in range(8):
        n = [int(x) for x in rng.integers(3, 40, 3)]
        res = 0.25 if corner else float(rng.uniform(0.02, 0.3))
        grid = Grid(n[0], n[1], n[2], res, (0.0, 0.0, 0.0) if corner else tuple(rng.uniform(-1, 1, 3)))
        ext = grid.extent
        centre = np.array(grid.origin) + ext / 2
        if corner:
            c = np.array([float(rng.integers(0, k)) for k in n]) * res
            target = c + res * rng.choice([-1.0, 1.0], 3)
        else:
            c = centre + rng.normal(0, 1.0, 3) * (np.linalg.norm(ext) if trial % 2 else 0.2 * np.linalg.norm(ext))
            target = centre + rng.normal(0, 0.3, 3) * ext
        cam = Camera(int(rng.integers(1, 50)), int(rng.integers(1, 40)), float(rng.uniform(10, 80)),
                     float(rng.uniform(10, 80)), float(rng.uniform(0, 40)), float(rng.uniform(0, 30)),
                     look_at(c, target))
        depth = rng.uniform(0.01, 3 * np.linalg.norm(ext), (cam.H, cam.W)).astype(np.float32)
        depth[rng.random(depth.shape) < 0.2] = 0.0
        depth[rng.random(depth.shape) < 0.05] = np.inf
        lut = noise_table(int(rng.integers(2, 100)), grid.diagonal * float(rng.uniform(0.5, 2)))

        class W:
            pass
        w = W()
        w.grid, w.prior, w.lut, w.iters = grid, 0.5, lut, 2
        from synth.scenes import Frame
        w.frames = [Frame(depth, cam)]
        mp = run_map(m, w, iters=2)
        _check_traversal(mp, oracle.trace_frames(grid, w.frames, lut))
        mp.close()


@pytest.mark.parametrize("name", ["room_small", "plain_64x48", "diff_small"])
def test_sensor_likelihood_matches_oracle(m, name):
    w = make_workload(name)
    mp = run_map(m, w, iters=0)
    nu32 = mp.export_nu().cpu().numpy()
    nu = nu32.astype(np.float64)
    ref = oracle.trace_frames(w.grid, w.frames, w.lut)
    ln = oracle.log_nu_edges(w.lut, ref["ray_off"], ref["Z"], ref["d"])
    np.testing.assert_allclose(nu, np.exp(ln), rtol=2e-5, atol=0)
    # edges far from their ray's measured range skip the FP64 evaluation and store the floor: exactly
    # the float the evaluation rounds to there, and most edges of a ray are such edges
    fl = np.float32(np.float64(w.lut.outlier_w) / np.float64(w.lut.d_hi))
    far = nu32 == fl
    assert far.mean() > 0.5
    assert np.array_equal(np.exp(ln[far]).astype(np.float32), nu32[far])
    mp.close()


def test_bias_table_matches_oracle(m):
    """A sensor-bias table (Section IV-C) shifts every likelihood's mean; both sides apply it alike."""
    import dataclasses
    w0 = make_workload("room_small")
    k = np.arange(w0.lut.n_bins)
    bias = (0.004 * np.sin(0.7 * k) + 0.002).astype(np.float32)
    w = dataclasses.replace(w0, lut=dataclasses.replace(w0.lut, bias=bias))
    mp = run_map(m, w)
    nu = mp.export_nu().cpu().numpy().astype(np.float64)
    ref = oracle.trace_frames(w.grid, w.frames, w.lut)
    ln = oracle.log_nu_edges(w.lut, ref["ray_off"], ref["Z"], ref["d"])
    np.testing.assert_allclose(nu, np.exp(ln), rtol=2e-5, atol=0)
    ln0 = oracle.log_nu_edges(w0.lut, ref["ray_off"], ref["Z"], ref["d"])
    assert np.max(np.abs(ln - ln0)) > 1.0          # the bias moves the likelihoods
    p = mp.marginals().cpu().numpy().astype(np.float64).ravel()
    ref = oracle.infer(w)
    check_marginals(p, ref["p"], workload_sensitivity(w, ref), "bias table")
    mp.close()


# --------------------------------------------------------------------------
# transpose
# --------------------------------------------------------------------------
def test_transpose_matches_stable_counting_sort(m):
    """Per voxel, the library's edge list equals the oracle's (edge-id order); voxels come in the
    library's internal order (8^3 bricks x-fastest, Morton order inside a brick)."""
    w = make_workload("room_small")
    mp = run_map(m, w, iters=0)
    tr = mp.export_transpose()
    ref = oracle.trace_frames(w.grid, w.frames, w.lut)
    vstart, eid = oracle.transpose(ref["vox"], w.grid.n_voxels)
    nonempty = np.nonzero(np.diff(vstart))[0]
    seg_vox = tr["seg_vox"].cpu().numpy().view(np.uint32).astype(np.int64)
    seg_off = tr["seg_off"].cpu().numpy().view(np.uint32).astype(np.int64)
    perm = tr["perm"].cpu().numpy().view(np.uint32).astype(np.int64)
    keys = voxel_key(seg_vox, w.grid)
    assert np.all(np.diff(keys) > 0)                      # strictly increasing internal keys
    order = np.argsort(seg_vox, kind="stable")
    np.testing.assert_array_equal(seg_vox[order], nonempty)
    lens = np.diff(seg_off)
    np.testing.assert_array_equal(lens[order], np.diff(vstart)[nonempty])
    regrouped = np.concatenate([perm[seg_off[s]:seg_off[s + 1]] for s in order])
    np.testing.assert_array_equal(regrouped, eid)
    assert mp.stats()["n_touched"] == len(nonempty)
    mp.close()


def test_group_tables_match_their_definition(m):
    """The per-tile voxel groups, bit for bit against their definition over the oracle's edges:
    tiles of whole rays within a 2048-edge window; per tile the edges sorted by (internal voxel
    key, edge); group ends, offsets, indices and keys.  Half of one frame's pixels see a near
    surface, so that tiles of more than 64 short rays (the sort path) sit beside tiles of a few
    long rays (the brick-mask path)."""
    from synth.scenes import Frame
    w = make_workload("room_small")
    near = w.frames[1].depth.copy()
    near[:, : near.shape[1] // 2] *= 0.05
    frames = [w.frames[0], Frame(near, w.frames[1].cam)]
    mp = run_map(m, w, frames=frames, iters=0)
    ref = oracle.trace_frames(w.grid, frames, w.lut)
    ro = ref["ray_off"]
    key = voxel_key(ref["vox"].astype(np.int64), w.grid)
    g = {k: v.cpu().numpy() for k, v in mp.export_groups().items()}
    E = len(key)
    tE = g["tile_E"]
    nt = len(tE) - 1
    assert tE[0] == 0 and tE[-1] == E and np.all(np.diff(tE) > 0)
    assert np.all(np.isin(tE, ro))                                  # whole rays
    assert np.all(tE[1:] - (tE[:-1] & ~7) <= 2048)                  # within the window
    nonempty = np.diff(ro) > 0
    starts = ro[:-1][nonempty]
    rays_per_tile = np.bincount(np.searchsorted(tE, starts, side="right") - 1, minlength=nt)
    assert rays_per_tile.max() > 64 and rays_per_tile.min() <= 64   # both paths
    tile = np.repeat(np.arange(nt), np.diff(tE))
    order = np.lexsort((np.arange(E), key, tile))                   # tile, voxel key, edge
    base = tE[:-1] & ~7
    np.testing.assert_array_equal(g["lidx"].view(np.uint16).astype(np.int64), order - base[tile[order]])
    ks, ts = key[order], tile[order]
    end = np.ones(E, bool)
    end[:-1] = (ks[1:] != ks[:-1]) | (ts[1:] != ts[:-1])
    bits = np.unpackbits(g["ends"].view(np.uint8), bitorder="little")[:E].astype(bool)
    np.testing.assert_array_equal(bits, end)
    start = np.r_[True, end[:-1]]
    tg = np.zeros(nt + 1, np.int64)
    tg[1:] = np.cumsum(np.bincount(ts[start], minlength=nt))
    np.testing.assert_array_equal(g["tg_off"], tg)
    gid = np.empty(E, np.int64)
    gid[order] = np.cumsum(start) - 1 - tg[ts]
    np.testing.assert_array_equal(g["gid"].view(np.uint16).astype(np.int64), gid)
    np.testing.assert_array_equal(g["gkey"].view(np.uint32).astype(np.int64), ks[start])
    assert mp.plan_info()["n_groups"] == tg[-1]
    mp.close()


def voxel_key(lin, grid):
    """Internal voxel key of linear voxel indices (8^3 bricks numbered x-fastest, Morton inside)."""
    lin = np.asarray(lin, np.int64)
    x, y, z = lin % grid.nx, (lin // grid.nx) % grid.ny, lin // (grid.nx * grid.ny)
    nbx, nby = (grid.nx + 7) // 8, (grid.ny + 7) // 8
    brick = (x >> 3) + nbx * ((y >> 3) + nby * (z >> 3))
    mort = np.zeros_like(lin)
    for bit in range(3):
        mort |= ((x >> bit) & 1) << (3 * bit) | ((y >> bit) & 1) << (3 * bit + 1) | ((z >> bit) & 1) << (3 * bit + 2)
    return (brick << 9) | mort


# --------------------------------------------------------------------------
# whole inference
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["plain_64x48", "room_small"])
@pytest.mark.parametrize("variant", ["default", "init_0.1", "nu_bg_0"])
def test_marginals_fp32_match_oracle(m, name, variant):
    w = make_workload(name)
    opt, kw = {}, {}
    if variant == "init_0.1":
        opt["init_p"], kw["init_p"] = 0.1, 0.1
    if variant == "nu_bg_0":
        opt["nu_bg"], kw["log_nu_bg"] = 0.0, -math.inf
    mp = run_map(m, w, **opt)
    p = mp.marginals().cpu().numpy().ravel().astype(np.float64)
    ref = oracle.infer(w, **kw)
    # well-conditioned cases: 1e-4 on every voxel; where loopy BP amplifies rounding
    # (test_conditioning.py) a bar scaled by the oracle's own sensitivity; every pass is
    # also checked exactly by test_every_pass_from_gpu_state
    check_marginals(p, ref["p"], workload_sensitivity(w, ref, **kw), f"{name} {variant}")
    mp.close()


@pytest.mark.parametrize("plan", [
    {},                                              # pipelined ray kernel, (tile, voxel) partials
    {"MRF_GROUPS": "0"},                             # pipelined, per-edge voxel totals
    {"MRF_RAY_ITEMS": "16"},                         # 4096-edge tiles, partials
    {"MRF_RAY_ITEMS": "16", "MRF_GROUPS": "0"},
    {"MRF_RAY_ITEMS": "16", "MRF_PIPE_THREADS": "128"},   # 128 threads x 16 edges, 2048-edge tiles
    {"MRF_RAY_PIPE": "0"},                           # standalone tile-per-CTA ray kernel
    {"MRF_RAY_ITEMS": "32"},                         # 8192-edge tiles (standalone only)
])
def test_kernel_plans_match_oracle(m, monkeypatch, plan):
    """Every ray-kernel plan the library can choose gives the oracle's marginals."""
    for k, v in plan.items():
        monkeypatch.setenv(k, v)
    w = make_workload("room_small")
    mp = run_map(m, w)
    info = mp.plan_info()
    kt = int(plan.get("MRF_RAY_ITEMS", "8"))
    assert info["ray_items"] == kt and info["n_ray_tiles"] > 0
    grouped = kt in (8, 16) and plan.get("MRF_RAY_PIPE", "1") != "0" and plan.get("MRF_GROUPS", "1") != "0"
    E = mp.stats()["n_edges"]
    if grouped:
        assert 0 < info["n_groups"] < E
    else:
        assert info["n_groups"] == 0
    p = mp.marginals().cpu().numpy().ravel().astype(np.float64)
    ref = oracle.infer(w)
    check_marginals(p, ref["p"], _room_small_sensitivity(w, ref), f"plan {plan}")
    mp.close()


_SENS = {}


def _room_small_sensitivity(w, ref):
    """The oracle's sensitivity on the 4-frame room (default options), computed once."""
    if "room_small" not in _SENS:
        _SENS["room_small"] = workload_sensitivity(w, ref)
    return _SENS["room_small"]


# first-pass messages as the library receives them (float32), so both sides start from one cavity
PASS_VARIANTS = {"default": {}, "init_0.1": {"init_p": 0.1}, "nu_bg_0": {"nu_bg": 0.0},
                 "init_sat": {"init_p": float(np.float32(1 - 1e-6))}, "init_free": {"init_p": float(np.float32(1e-6))}}


@pytest.mark.parametrize("name,variant", [("plain_64x48", "nu_bg_0"), ("room_small", "init_0.1"),
                                          ("room_small", "default"), ("room_small", "init_sat"),
                                          ("plain_64x48", "init_free")])
def test_every_pass_from_gpu_state(m, name, variant):
    """Pass t of the GPU equals the oracle's pass t applied to the GPU's own state after pass t-1.

    init_sat starts every edge at cavity log-odds +13.8 (odds 1e6): along a ray the forward state
    (c + A') / P of the floored kernels grows by 1e6 per voxel and overflows to infinity within a
    few voxels, the path where the messages must go to their limit 0; init_free starts at -13.8."""
    w = make_workload(name)
    opt = PASS_VARIANTS[variant]
    ref = oracle.trace_frames(w.grid, w.frames, w.lut)
    ro, vox = ref["ray_off"], ref["vox"].astype(np.int64)
    mp = run_map(m, w, iters=0, **opt)
    nu = mp.export_nu().cpu().numpy().astype(np.float64)
    lbg = -math.inf if variant == "nu_bg_0" else oracle.default_log_nu_bg(w.lut)
    init = opt.get("init_p", w.prior)
    lp = math.log(w.prior) - math.log1p(-w.prior)
    lam_prev = T_prev = None
    for t in range(1, w.iters + 1):
        mp.infer(t)
        lam32, T32 = (x.cpu().numpy() for x in mp.export_messages())
        lam, T = lam32.astype(np.float64), T32.astype(np.float64)
        # the cavity is the FP32 difference of the stored FP32 values, on both sides
        L = np.full(len(vox), np.float64(np.float32(math.log(init) - math.log1p(-init)))) if t == 1 else \
            (T_prev[vox] - lam_prev).astype(np.float64)
        lam_ref = np.zeros(len(vox))
        for r in range(len(ro) - 1):
            a, b = ro[r], ro[r + 1]
            if b > a:
                lam_ref[a:b] = oracle.ray_messages(L[a:b], np.log(nu[a:b]), lbg)
        assert np.max(np.abs(lam - lam_ref) / (1 + np.abs(lam_ref))) <= 2e-5, t
        T_ref = lp + np.bincount(vox, weights=lam, minlength=w.grid.n_voxels)
        bound = 1e-5 * (1 + np.bincount(vox, weights=np.abs(lam), minlength=w.grid.n_voxels))
        assert np.all(np.abs(T - T_ref) <= bound), t
        lam_prev, T_prev = lam32, T32
    mp.close()


def test_marginals_fp64_match_oracle(m):
    for name in ["plain_64x48", "room_small"]:
        w = make_workload(name)
        mp = run_map(m, w, precision=m.PREC_F64)
        p = mp.marginals().cpu().numpy()
        lam, T = mp.export_messages()
        ref = oracle.infer(w)
        # marginals leave the library as float32; compare T in FP64
        Tref = ref["T"]
        Tg = T.cpu().numpy()
        dT = np.abs(Tg - Tref) / (1 + np.abs(Tref))
        assert dT.max() <= P_TOL_F64, (name, dT.max())
        pv = 1 / (1 + np.exp(-Tg))
        assert np.abs(pv - ref["p"]).max() <= P_TOL_F64
        assert np.abs(p.ravel() - ref["p"]).max() <= 1e-6
        mp.close()


def test_iteration_counts_and_untouched_voxels(m):
    w = make_workload("room_small")
    ref_csr = oracle.trace_frames(w.grid, w.frames, w.lut)
    touched = np.zeros(w.grid.n_voxels, bool)
    touched[ref_csr["vox"]] = True
    for iters in [0, 1, 2, 5]:
        mp = run_map(m, w, iters=iters)
        p = mp.marginals().cpu().numpy().ravel().astype(np.float64)
        if iters == 0:
            assert np.all(p == np.float32(w.prior))
        assert np.all(p[~touched] == np.float32(w.prior))
        ref = oracle.infer(w, iters=iters)
        assert np.abs(p - ref["p"]).max() <= P_TOL_F32
        mp.close()


def test_bitwise_deterministic(m):
    w = make_workload("room_small")
    a = run_map(m, w)
    b = run_map(m, w)
    pa, pb = a.marginals().cpu().numpy(), b.marginals().cpu().numpy()
    assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
    la, _ = a.export_messages()
    a.infer(w.iters)   # re-running infer restarts from the initial messages
    lb, _ = a.export_messages()
    assert torch.equal(la, lb)
    a.close()
    b.close()


def test_empty_and_degenerate_frames(m):
    w = make_workload("plain_64x48")
    fr = w.frames[0]
    mp = m.Map(w.grid, w.prior)
    mp.infer(3)  # no frames at all
    assert torch.all(mp.marginals() == np.float32(w.prior))
    mp.add_frame(torch.zeros(5, 7, device="cuda"), fr.cam.pose, fr.cam, w.lut)  # every pixel invalid
    mp.infer(3)
    assert mp.stats()["n_edges"] == 0
    assert torch.all(mp.marginals() == np.float32(w.prior))
    # one valid pixel
    d = np.zeros_like(fr.depth)
    d[24, 32] = fr.depth[24, 32]
    mp.add_frame(torch.from_numpy(d).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(4)
    p = mp.marginals().cpu().numpy().ravel().astype(np.float64)
    class W:
        pass
    w1 = W()
    w1.grid, w1.prior, w1.lut, w1.iters = w.grid, w.prior, w.lut, 4
    from synth.scenes import Frame
    ref = oracle.infer(w1, frames=[Frame(d, fr.cam)])  # the all-invalid frame adds no edges
    assert np.abs(p - ref["p"]).max() <= P_TOL_F32
    mp.close()


def test_reset_and_host_entry_points(m):
    w = make_workload("plain_64x48")
    fr = w.frames[0]
    mp = m.Map(w.grid, w.prior)
    mp.add_frame(fr.depth, fr.cam.pose, fr.cam, w.lut)        # host depth
    mp.infer(w.iters)
    p_host = mp.marginals_host().ravel()
    mp.reset()
    assert mp.stats()["n_edges"] == 0
    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters)
    p_dev = mp.marginals().cpu().numpy().ravel()
    assert np.array_equal(p_host, p_dev)
    mp.close()


def test_errors_are_sticky_and_reported(m):
    w = make_workload("plain_64x48")
    fr = w.frames[0]
    mp = m.Map(w.grid, w.prior)
    with pytest.raises(m.MRFError) as ei:
        mp.infer(-1)
    assert ei.value.code == m.MRF_EINVAL and "iters" in str(ei.value)
    bad = type(w.lut)(1, 0.0, 1.0, np.zeros(1, np.float32), 0.0)
    with pytest.raises(m.MRFError):
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, bad)
    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)  # cleared by the report
    mp.close()


# --------------------------------------------------------------------------
# standalone kernels on caller buffers: ragged rays, many tiles, edge cases
# --------------------------------------------------------------------------
def _random_rays(rng, R, max_len, empty_frac=0.1):
    N = rng.integers(1, max_len + 1, R)
    N[rng.random(R) < empty_frac] = 0
    N[rng.integers(0, R, 3)] = max_len
    off = np.zeros(R + 1, np.int64)
    np.cumsum(N, out=off[1:])
    return off


@pytest.mark.parametrize("max_len,R", [(1, 5000), (7, 3000), (60, 2000), (450, 600), (1500, 200), (5000, 40)])
@pytest.mark.parametrize("first", [0, 1])
@pytest.mark.parametrize("nu_bg", [0.0, 0.00225, 3.0])
def test_ray_messages_kernel(m, max_len, R, first, nu_bg):
    rng = np.random.default_rng(max_len * 7 + R + first)
    off = _random_rays(rng, R, max_len)
    E = int(off[-1])
    V = 1000
    vox = rng.integers(0, V, E).astype(np.int32)
    nu = np.exp(rng.uniform(-6, 5, E)).astype(np.float32)
    T = rng.uniform(-15, 15, V).astype(np.float32)
    lam_old = rng.uniform(-8, 8, E).astype(np.float32)
    L0 = -2.1972246
    lam = torch.from_numpy(lam_old.copy()).cuda()
    m.ray_messages(torch.from_numpy(off).cuda(), torch.from_numpy(vox).cuda(), torch.from_numpy(nu).cuda(),
                   torch.from_numpy(T).cuda(), lam, nu_bg, bool(first), L0)
    got = lam.cpu().numpy().astype(np.float64)
    lbg = math.log(nu_bg) if nu_bg > 0 else -math.inf
    ref = np.zeros(E)
    L_all = np.full(E, np.float64(np.float32(L0))) if first else \
        (T.astype(np.float64)[vox] - lam_old.astype(np.float64))
    for r in range(R):
        a, b = off[r], off[r + 1]
        if b > a:
            ref[a:b] = oracle.ray_messages(L_all[a:b], np.log(nu[a:b].astype(np.float64)), lbg)
    err = np.abs(got - ref) / (1 + np.abs(ref))
    assert err.max() <= 2e-5, (err.max(), np.argmax(err))


def test_ray_messages_kernel_rejects_overlong_rays(m):
    off = torch.tensor([0, 9000], dtype=torch.int64, device="cuda")
    z = torch.zeros(9000, device="cuda")
    with pytest.raises(m.MRFError):
        m.ray_messages(off, torch.zeros(9000, dtype=torch.int32, device="cuda"), z + 1, z, z.clone(), 0.1)


@pytest.mark.parametrize("E,V", [(1, 1), (4095, 3), (4096, 1), (4097, 2), (300_000, 1), (300_000, 50_000),
                                 (1_000_003, 2_000_000)])
def test_voxel_reduce_kernel(m, E, V):
    rng = np.random.default_rng(E + V)
    vox = rng.integers(0, V, E)
    if V > 1:   # one heavy voxel spanning many tiles, as the camera voxel of a frame does
        vox[rng.random(E) < 0.3] = V // 2
    lam = rng.uniform(-6, 6, E).astype(np.float32)
    order = np.argsort(vox, kind="stable")
    sk = vox[order]
    heads = np.nonzero(np.r_[True, sk[1:] != sk[:-1]])[0]
    seg_off = np.append(heads, E).astype(np.int32)
    seg_vox = sk[heads].astype(np.int32)
    T = torch.full((V,), 123.0, device="cuda")
    m.voxel_reduce(torch.from_numpy(order.astype(np.int32)).cuda(), torch.from_numpy(seg_off).cuda(),
                   torch.from_numpy(seg_vox).cuda(), torch.from_numpy(lam).cuda(), 0.25, T)
    ref = np.full(V, 123.0)
    sums = np.add.reduceat(lam.astype(np.float64)[order], heads)
    abs_sums = np.add.reduceat(np.abs(lam.astype(np.float64))[order], heads)
    ref[seg_vox] = 0.25 + sums
    got = T.cpu().numpy().astype(np.float64)
    bound = np.full(V, 0.0)
    bound[seg_vox] = 1e-5 * (1 + abs_sums)
    assert np.all(np.abs(got - ref) <= bound + 1e-6)
