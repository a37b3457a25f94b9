"""mrf_voxel_reduce_noalloc: the voxel totals with the library's own static
scratch, for callers that cannot allocate device memory during a call.

Checked through the C ABI against mrf_voxel_reduce (caller-provided
workspace) on the same inputs, for two calls in a row (the scratch keeps the
previous call's contents), plus the size limit.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _segments(rng, E, V):
    vox = rng.integers(0, V, E)
    vox[rng.random(E) < 0.3] = V // 2            # one voxel spanning many 4096-edge tiles
    order = np.argsort(vox, kind="stable")
    sk = vox[order]
    heads = np.nonzero(np.r_[True, sk[1:] != sk[:-1]])[0]
    return order.astype(np.int32), np.append(heads, E).astype(np.int32), sk[heads].astype(np.int32)


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice():
    import paper_2006_03512_gb300 as m
    m.build()
    for call, (E, V) in enumerate([(300_000, 50_000), (1_000_003, 7)]):
        rng = np.random.default_rng(call)
        perm, seg_off, seg_vox = _segments(rng, E, V)
        lam = rng.uniform(-6, 6, E).astype(np.float32)
        d = {k: torch.from_numpy(v).cuda() for k, v in
             dict(perm=perm, seg_off=seg_off, seg_vox=seg_vox, lam=lam).items()}
        T_ref = torch.full((V,), -3.0, device="cuda")
        m.voxel_reduce(d["perm"], d["seg_off"], d["seg_vox"], d["lam"], 0.25, T_ref)
        T_na = torch.full((V,), -3.0, device="cuda")
        m.voxel_reduce_noalloc(d["perm"], d["seg_off"], d["seg_vox"], d["lam"], 0.25, T_na)
        torch.cuda.synchronize()
        abs_sum = np.zeros(V)
        np.add.at(abs_sum, seg_vox, np.add.reduceat(np.abs(lam.astype(np.float64))[perm], seg_off[:-1]))
        tol = torch.from_numpy(1e-5 * (1 + abs_sum)).cuda()
        assert bool(((T_na.double() - T_ref.double()).abs() <= tol).all()), call


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2006_03512_gb300 as m
    m.build()
    L = m.lib()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = L.mrf_voxel_reduce_noalloc(p, p, p, 1, m.NOALLOC_MAX_EDGES + 1, p, ctypes.c_float(0.0), p, None)
    assert rc == m.MRF_ERANGE
