"""Conditioning of loopy BP on the parity workloads (FP64 oracle only, CPU).

Loopy BP has no contraction guarantee (Section III-B notes convergence is not
guaranteed).  These tests measure how far the FP64 oracle's marginals move
when its inputs get a perturbation the size of FP32 rounding (1e-7 relative
noise on the sensor likelihoods).  Where that alone moves a marginal by more
than 5e-6, a bitwise-different FP32 implementation cannot be held to 1e-4 on
every voxel, and the GPU parity test uses a bar scaled by this sensitivity.
"""
import numpy as np
import pytest

import oracle
from synth import make_workload


def sensitivity(w, init_p, iters, seed=0):
    csr = oracle.trace_frames(w.grid, w.frames, w.lut)
    ln = oracle.log_nu_edges(w.lut, csr["ray_off"], csr["Z"], csr["d"])
    lbg = oracle.default_log_nu_bg(w.lut)
    _, _, p0 = oracle.bp(csr["ray_off"], csr["vox"], ln, w.grid.n_voxels, w.prior, init_p, lbg, iters)
    rng = np.random.default_rng(seed)
    _, _, p1 = oracle.bp(csr["ray_off"], csr["vox"], ln + rng.normal(0, 1e-7, len(ln)), w.grid.n_voxels, w.prior,
                         init_p, lbg, iters)
    return np.abs(p1 - p0)


def test_single_frame_default_is_well_conditioned():
    w = make_workload("plain_64x48")
    d = sensitivity(w, w.prior, w.iters)
    assert d.max() < 5e-6


def test_room_default_amplifies_rounding_on_a_few_voxels():
    w = make_workload("room_small")
    d = sensitivity(w, w.prior, w.iters)
    assert d.max() > 5e-6 and np.percentile(d, 99.9) < 1e-6


def test_paper_initialisation_on_room_is_ill_conditioned():
    """init_p = 0.1 (Section IV-A) on the 4-frame room: a few voxels move ~1e-4 under 1e-7 noise."""
    w = make_workload("room_small")
    d = sensitivity(w, 0.1, w.iters)
    assert d.max() > 1e-4
    assert np.percentile(d, 99.9) < 1e-6
