"""Parity at full size: 30 frames of 640x480 over a 256^3 grid, 20 passes (the room), and 60 frames
of 424x240 over a 512x512x256 grid, 30 passes, with rays up to ~700 voxels (the corridor).

The oracle cannot run the whole loopy BP at this size in a test, so it checks
what it can compute piece by piece, in the launch configuration the bench
times:
  * traversal of three whole frames, bit-exact;
  * the transpose: a stable sort of the edges by voxel (checked on the GPU);
  * one BP pass on sampled rays: the ray->voxel messages of pass t+1 from the
    GPU's own pass-t state, recomputed by the oracle;
  * voxel totals of sampled voxels from the GPU's messages, summed in FP64;
  * invariants: p in [0, 1], untouched voxels keep the prior, determinism.
"""
import math

import numpy as np
import pytest

import oracle
from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def u32(t):
    """The library's uint32 arrays arrive in int32 tensors; widen without sign extension."""
    return t.long() & 0xFFFFFFFF


def key_of(lin, grid):
    """Internal voxel key (8^3 bricks x-fastest, Morton order inside) of linear voxel indices."""
    x, y, z = lin % grid.nx, (lin // grid.nx) % grid.ny, lin // (grid.nx * grid.ny)
    nbx, nby = (grid.nx + 7) // 8, (grid.ny + 7) // 8
    key = ((x >> 3) + nbx * ((y >> 3) + nby * (z >> 3))) << 9
    for bit in range(3):
        key |= ((x >> bit) & 1) << (3 * bit) | ((y >> bit) & 1) << (3 * bit + 1) | ((z >> bit) & 1) << (3 * bit + 2)
    return key


@pytest.fixture(scope="module", params=["room_30x640x480", "corridor_60x424x240"])
def full(request):
    import paper_2006_03512_gb300 as m
    m.build()
    w = make_workload(request.param)
    mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p))
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    yield m, w, mp
    mp.close()


def test_fullsize_traversal_three_frames(full):
    m, w, mp = full
    ex = mp.export_rays()
    ro = ex["ray_off"].cpu().numpy()
    npix = w.frames[0].cam.W * w.frames[0].cam.H
    nf = len(w.frames)
    for f in [0, nf // 2 - 2, nf - 1]:
        ref = oracle.trace_frame(w.grid, w.frames[f].cam, w.frames[f].depth, w.lut)
        a, b = ro[f * npix], ro[(f + 1) * npix]
        np.testing.assert_array_equal(ro[f * npix:(f + 1) * npix + 1] - a, ref["ray_off"])
        np.testing.assert_array_equal(ex["vox"][a:b].cpu().numpy().view(np.uint32), ref["vox"])
        np.testing.assert_array_equal(ex["d"][a:b].cpu().numpy().view(np.uint32), ref["d"].view(np.uint32))


def test_fullsize_transpose_is_stable_sort(full):
    m, w, mp = full
    tr = mp.export_transpose()
    # voxel keys (< 2^24 here, so int32) and the permutation, checked in chunks
    # so that no temporary spans all 2.6e9 edges in int64
    vox = mp.export_rays()["vox"]
    E = vox.numel()
    chunk = 1 << 27
    for a in range(0, E, chunk):
        vox[a:a + chunk] = key_of(vox[a:a + chunk], w.grid)
    perm32 = tr["perm"]
    seen = torch.zeros(E, dtype=torch.bool, device="cuda")
    for a in range(0, E, chunk):
        b = min(E, a + chunk + 1)                      # one position of overlap
        perm = u32(perm32[a:b])
        keys = vox[perm]
        assert bool((keys[1:] >= keys[:-1]).all())
        same = keys[1:] == keys[:-1]
        assert bool((perm[1:][same] > perm[:-1][same]).all())      # stable
        seen[perm] = True
        del perm, keys, same
    assert bool(seen.all())                                          # a permutation
    del seen
    seg_off = u32(tr["seg_off"])
    assert int(seg_off[0]) == 0 and int(seg_off[-1]) == E
    heads = u32(perm32[seg_off[:-1]])
    assert torch.equal(vox[heads], key_of(tr["seg_vox"], w.grid))


def test_fullsize_one_pass_on_sampled_rays_and_voxels(full):
    m, w, mp = full
    t = w.iters - 1
    mp.infer(t)
    lam_t, T_t = mp.export_messages()
    lam_t, T_t = lam_t.clone(), T_t.clone()
    mp.infer(t + 1)
    lam_n, T_n = mp.export_messages()
    ex = mp.export_rays()
    ro = ex["ray_off"].cpu().numpy()
    nu = mp.export_nu()
    rng = np.random.default_rng(7)
    R = len(ro) - 1
    rays = [r for r in rng.integers(0, R, 4000) if ro[r + 1] > ro[r]][:1500]
    n = np.diff(ro)
    rays += [int(r) for r in np.flatnonzero(n > 512)[:300]]      # the longest rays, if any
    rays.append(int(np.argmax(n)))
    lbg = oracle.default_log_nu_bg(w.lut)
    worst = 0.0
    for r in rays:
        a, b = int(ro[r]), int(ro[r + 1])
        vx = u32(ex["vox"][a:b])
        L = (T_t[vx].double() - lam_t[a:b].double()).cpu().numpy()
        ref = oracle.ray_messages(L, np.log(nu[a:b].double().cpu().numpy()), lbg)
        got = lam_n[a:b].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - ref) / (1 + np.abs(ref)))))
    assert worst <= 2e-5, worst
    # voxel totals of sampled non-empty voxels, summed in FP64 from the GPU's messages
    tr = mp.export_transpose()
    seg_off = u32(tr["seg_off"])
    S = tr["seg_vox"].numel()
    sample = torch.from_numpy(rng.integers(0, S, 5000)).cuda()
    sample = torch.cat([sample, torch.argmax(seg_off[1:] - seg_off[:-1]).view(1)])  # the heaviest voxel
    lp = math.log(w.prior) - math.log1p(-w.prior)
    perm = u32(tr["perm"])
    for s in sample.tolist():
        a, b = int(seg_off[s]), int(seg_off[s + 1])
        vals = lam_n[perm[a:b]].double()
        ref = lp + float(vals.sum())
        got = float(T_n[int(tr["seg_vox"][s])])
        assert abs(got - ref) <= 1e-5 * (1 + float(vals.abs().sum())), (s, got, ref)


def test_fullsize_invariants_and_determinism(full):
    m, w, mp = full
    mp.infer(w.iters)
    p1 = mp.marginals()
    lam1, _ = mp.export_messages()
    lam1 = lam1.clone()
    mp.infer(w.iters)
    p2 = mp.marginals()
    lam2, _ = mp.export_messages()
    assert torch.equal(p1, p2) and torch.equal(lam1, lam2)
    assert bool(((p1 >= 0) & (p1 <= 1)).all())
    touched = torch.zeros(w.grid.n_voxels, dtype=torch.bool, device="cuda")
    touched[u32(mp.export_transpose()["seg_vox"])] = True
    assert bool((p1.view(-1)[~touched] == np.float32(w.prior)).all())
    # the map is not the trivial fixed point: free space is carved and
    # surfaces are found (tens of thousands and about a thousand voxels)
    assert int((p1 < 0.1).sum()) > 10_000 and int((p1 > 0.9).sum()) > 500
    st = mp.stats()
    fr = w.frames[0]
    assert st["n_edges"] > 10 ** 9 and st["n_rays"] == len(w.frames) * fr.cam.W * fr.cam.H


@pytest.mark.parametrize("name", ["room_30x640x480", "corridor_60x424x240"])
def test_frame0_whole_bp_matches_oracle(name):
    """Whole loopy BP at the benchmarked geometry: the first frame of each full-size workload (full
    grid, the workload's passes and first-pass message), every voxel's marginal against the FP64
    oracle's.  The bars follow the oracle's own measured response to rounding-size noise on its
    likelihoods (loopy BP has no convergence guarantee, Section III-B):
      FP64 on the GPU: p within 1e-9 on every voxel the oracle's FP64-size probe (1e-15 relative
        noise) moves by at most 1e-12; elsewhere within 100 x that probe's movement;
      FP32: 1e-4 on every voxel the oracle's FP32-size probes (1e-7 relative noise on the
        likelihoods; the first-pass log-odds one float32 ulp up) move by at most 5e-6
        (parity_bars.py); the count and size of the misses elsewhere are printed.
    The oracle runs with the first-pass message the library received (the ABI's float)."""
    from parity_bars import WELL_CONDITIONED, sensitivity_map
    import paper_2006_03512_gb300 as m
    m.build()
    w = make_workload(name)
    fr = w.frames[0]
    ip = float(np.float32(w.init_p or w.prior))   # mrf_options.init_p is a float
    ref = oracle.infer(w, init_p=ip, frames=[fr])
    args = (ref["csr"]["ray_off"], ref["csr"]["vox"], ref["log_nu"], w.grid.n_voxels, w.prior, ip,
            oracle.default_log_nu_bg(w.lut), w.iters, ref["p"])
    sens32 = sensitivity_map(*args)
    rng = np.random.default_rng(1)
    p64 = oracle.bp(*args[:2], args[2] + rng.normal(0, 1e-15, len(args[2])), *args[3:8])[2]
    sens64 = np.abs(p64 - ref["p"])
    for prec in (m.PREC_F64, m.PREC_F32):
        mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p, precision=prec))
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
        mp.infer(w.iters)
        assert mp.stats()["n_edges"] == int(ref["csr"]["ray_off"][-1])
        if prec == m.PREC_F64:
            _, T = mp.export_messages()
            p = 1 / (1 + np.exp(-T.cpu().numpy().astype(np.float64)))
            err = np.abs(p - ref["p"])
            well = sens64 <= 1e-12
            print(f"{name} frame 0 FP64: max {err.max():.3g}, voxels > 1e-9: {int((err > 1e-9).sum())}, "
                  f"probe-sensitive voxels {int((~well).sum())} (probe max {sens64.max():.3g}), "
                  f"max on the rest {err[well].max():.3g}")
            assert err[well].max() <= 1e-9, (name, float(err[well].max()))
            assert np.all(err <= np.maximum(1e-9, 100 * sens64)), (name, float(err.max()))
        else:
            p = mp.marginals().cpu().numpy().astype(np.float64).ravel()
            err = np.abs(p - ref["p"])
            well = sens32 <= WELL_CONDITIONED
            print(f"{name} frame 0 FP32: max {err.max():.3g}, voxels > 1e-4: {int((err > 1e-4).sum())}, "
                  f"probe-sensitive voxels {int((~well).sum())} (probe max {sens32.max():.3g}), "
                  f"max on the rest {err[well].max():.3g}")
            assert err[well].max() <= 1e-4, (name, float(err[well].max()))
        mp.close()
