"""Failure detection without a GPU fault: injected allocation failures and a bounded device-side wait that
times out.  Every failure comes back as a status code; the context stays usable and gives the same
marginals afterwards; a destroyed context returns its memory.
"""
import time

import numpy as np
import pytest

from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2006_03512_gb300 as m
    m.build()
    return m


def run(m, mp, w):
    for fr in w.frames:
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
    mp.infer(w.iters)
    return mp.marginals().clone()


def test_wait_probe_times_out_and_the_context_recovers(m):
    w = make_workload("room_small")
    mp = m.Map(w.grid, w.prior)
    p_ref = run(m, mp, w)
    mp.debug_wait_probe()
    t0 = time.perf_counter()
    with pytest.raises(m.MRFError) as ei:
        mp.synchronize()
    dt = time.perf_counter() - t0
    assert ei.value.code == m.MRF_ETIMEOUT and "gave up" in str(ei.value)
    assert 0.5 < dt < 60.0, dt
    mp.synchronize()                      # the condition was cleared
    mp.infer(w.iters)
    assert torch.equal(mp.marginals(), p_ref)
    mp.close()


def test_injected_allocation_failures_are_clean(m):
    w = make_workload("room_small")
    mp = m.Map(w.grid, w.prior)
    p_ref = run(m, mp, w)
    mp.close()
    # after one whole map's life, so that the kernels' code is loaded on the device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    for nth in range(1, 200):
        mp = m.Map(w.grid, w.prior)
        mp.debug_fail_alloc(nth)
        try:
            run(m, mp, w)
            hit = False
        except m.MRFError as e:
            assert e.code == m.MRF_ENOMEM and "injected" in str(e), e
            hit = True
        if hit:
            failures += 1
            # the same context, after the error was read, maps the same frames to the same marginals
            mp.reset()
            assert torch.equal(run(m, mp, w), p_ref)
        mp.close()
        if not hit:      # past the last allocation of the sequence
            break
    assert failures >= 10, failures
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20), (free0, free1)   # destroyed contexts gave their memory back
