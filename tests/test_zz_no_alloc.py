"""mrf_voxel_reduce_noalloc: the voxel totals with the library's own static
scratch, for callers that cannot allocate device memory during a call (a
mapping loop under a fixed memory budget, code inside an allocator's
callbacks).

Checked through the C ABI on two calls in a row, the larger first, so that the
second call runs over the first one's leftovers in the shared scratch:
  * against the FP64 host sum logit_prior + sum of lam[perm] over each voxel's
    segment, within 1e-5 (1 + sum |lam|) (FP32 accumulation of up to a million
    terms of |lam| <= 6, Kahan-compensated);
  * against mrf_voxel_reduce (caller-provided workspace) bitwise: both run the
    same kernels in the same order.
Plus the size limit.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _segments(rng, E, V, heavy):
    vox = rng.integers(0, V, E)
    vox[rng.random(E) < heavy] = V // 2          # one voxel spanning many 4096-edge tiles
    order = np.argsort(vox, kind="stable")
    sk = vox[order]
    heads = np.nonzero(np.r_[True, sk[1:] != sk[:-1]])[0]
    return order.astype(np.int32), np.append(heads, E).astype(np.int32), sk[heads].astype(np.int32)


@pytest.mark.gpu
def test_noalloc_matches_fp64_sums_and_allocating_entry_point_twice():
    import paper_2006_03512_gb300 as m
    m.build()
    prior = 0.25
    # larger call first (1M edges, a third of them in one voxel), then a smaller
    # one with another segment layout over what the first left in the scratch
    for call, (E, V, heavy) in enumerate([(1_000_003, 97, 0.35), (300_001, 50_000, 0.1)]):
        rng = np.random.default_rng(call + 11)
        perm, seg_off, seg_vox = _segments(rng, E, V, heavy)
        lam = rng.uniform(-6, 6, E).astype(np.float32)
        d = {k: torch.from_numpy(v).cuda() for k, v in
             dict(perm=perm, seg_off=seg_off, seg_vox=seg_vox, lam=lam).items()}
        T_na = torch.full((V,), -3.0, device="cuda")
        m.voxel_reduce_noalloc(d["perm"], d["seg_off"], d["seg_vox"], d["lam"], prior, T_na)
        T_ref = torch.full((V,), -3.0, device="cuda")
        m.voxel_reduce(d["perm"], d["seg_off"], d["seg_vox"], d["lam"], prior, T_ref)
        torch.cuda.synchronize()
        lam64 = lam.astype(np.float64)[perm]
        exact = np.full(V, -3.0)
        exact[seg_vox] = prior + np.add.reduceat(lam64, seg_off[:-1])
        abs_sum = np.zeros(V)
        abs_sum[seg_vox] = np.add.reduceat(np.abs(lam64), seg_off[:-1])
        t = T_na.double().cpu().numpy()
        err = np.abs(t - exact)
        assert (err <= 1e-5 * (1 + abs_sum)).all(), (call, float(err.max()))
        assert torch.equal(T_na, T_ref), call


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2006_03512_gb300 as m
    m.build()
    L = m.lib()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = L.mrf_voxel_reduce_noalloc(p, p, p, 1, m.NOALLOC_MAX_EDGES + 1, p, ctypes.c_float(0.0), p, None)
    assert rc == m.MRF_ERANGE
