"""Pins of the oracle's differentiation code (CPU): the held-out loss against
enumeration of every occupancy configuration, and each adjoint against
central differences of the forward it reverses.

The forward messages are the oracle's log-domain ray_messages; the adjoint is
a separate linear-domain restatement, so agreement is not circular.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from synth.scenes import NoiseTable

H = 1e-6


def _fd(f, x, i, h=H):
    xp, xm = x.copy(), x.copy()
    xp[i] += h
    xm[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


@pytest.mark.parametrize("N", [1, 2, 5, 12])
@pytest.mark.parametrize("nu_bg", [0.05, 1.7])
def test_ray_messages_adjoint_matches_central_differences(N, nu_bg):
    rng = np.random.default_rng(N * 10 + int(nu_bg * 10))
    L = rng.uniform(-4, 4, N)
    nu = np.exp(rng.uniform(-3, 3, N))
    g = rng.normal(size=N)

    def f_L(x):
        return float(g @ oracle.ray_messages(x, np.log(nu), math.log(nu_bg)))

    def f_nu(x):
        return float(g @ oracle.ray_messages(L, np.log(x), math.log(nu_bg)))

    def f_bg(x):
        return float(g @ oracle.ray_messages(L, np.log(nu), math.log(x[0])))

    gL, gnu, gbg = oracle.ray_messages_adjoint(L, nu, nu_bg, g)
    for i in range(N):
        assert abs(gL[i] - _fd(f_L, L, i)) <= 1e-6 * (1 + abs(gL[i])), i
        assert abs(gnu[i] - _fd(f_nu, nu, i)) <= 1e-6 * (1 + abs(gnu[i])), i
    assert abs(gbg - _fd(f_bg, np.array([nu_bg]), 0)) <= 1e-6 * (1 + abs(gbg))


def test_ray_messages_adjoint_stops_at_the_clamp():
    # a one-voxel ray with nu far above nu_bg: lambda = log(nu / nu_bg) > 64 is clamped
    gL, gnu, gbg = oracle.ray_messages_adjoint(np.array([0.0]), np.array([1e30]), 1e-5, np.array([1.0]))
    assert gL[0] == 0 and gnu[0] == 0 and gbg == 0


def _enumerated_S(p, nu, nu_bg):
    """sum over every occupancy configuration of its probability times the likelihood of the depth:
    nu of the first occupied voxel, nu_bg if none is occupied."""
    N = len(p)
    S = 0.0
    for o in itertools.product([0, 1], repeat=N):
        pr = np.prod([p[i] if o[i] else 1 - p[i] for i in range(N)])
        first = next((i for i in range(N) if o[i]), None)
        S += pr * (nu_bg if first is None else nu[first])
    return S


def _rays(rng, R, V, max_len):
    lens = rng.integers(1, max_len + 1, R)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vox = np.concatenate([rng.choice(V, n, replace=False) for n in lens]).astype(np.uint32)
    return off, vox


def test_heldout_loss_matches_enumeration():
    rng = np.random.default_rng(3)
    V = 12
    off, vox = _rays(rng, 6, V, 9)
    p = rng.uniform(0.02, 0.98, V)
    nu = np.exp(rng.uniform(-3, 3, off[-1]))
    nu_bg = 0.07
    ref = -sum(math.log(_enumerated_S(p[vox[off[r]:off[r + 1]]], nu[off[r]:off[r + 1]], nu_bg))
               for r in range(len(off) - 1))
    assert oracle.heldout_loss(off, vox, nu, nu_bg, p) == pytest.approx(ref, rel=1e-12)
    # certain occupancy: the first voxel is occupied for sure
    p1 = p.copy()
    p1[vox[0]] = 1.0
    S0 = nu[0]
    loss1 = oracle.heldout_loss(off[:2], vox[:off[1]], nu[:off[1]], nu_bg, p1)
    assert loss1 == pytest.approx(-math.log(S0), rel=1e-12)


def test_heldout_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    V = 15
    off, vox = _rays(rng, 8, V, 7)
    p = rng.uniform(0.05, 0.95, V)
    nu = np.exp(rng.uniform(-2, 2, off[-1]))
    nu_bg = 0.3
    loss, gp, gnu, gbg = oracle.heldout_loss(off, vox, nu, nu_bg, p, grad=True)
    for v in range(V):
        assert gp[v] == pytest.approx(_fd(lambda x: oracle.heldout_loss(off, vox, nu, nu_bg, x), p, v),
                                      rel=1e-6, abs=1e-9)
    for e in range(0, len(nu), 3):
        assert gnu[e] == pytest.approx(_fd(lambda x: oracle.heldout_loss(off, vox, x, nu_bg, p), nu, e),
                                       rel=1e-6, abs=1e-9)
    assert gbg == pytest.approx(_fd(lambda x: oracle.heldout_loss(off, vox, nu, x[0], p), np.array([nu_bg]), 0),
                                rel=1e-6)


def _tiny_problem(seed, R=40, Rh=12, V=25, max_len=8):
    """Rays over a small shared voxel set (so BP is loopy), ranges increasing along each ray and a measured
    range near each ray's end, with an 8-bin table over [0, 3] m."""
    rng = np.random.default_rng(seed)

    def csr(R_):
        off, vox = _rays(rng, R_, V, max_len)
        d = np.concatenate([np.cumsum(rng.uniform(0.05, 0.15, n)) + 0.3 for n in np.diff(off)]).astype(np.float32)
        Z = np.array([d[off[r + 1] - 1] + rng.normal(0, 0.05) for r in range(R_)], np.float32)
        return dict(ray_off=off, vox=vox, d=d, Z=Z)

    lut = NoiseTable(8, 0.0, 3.0, np.log(rng.uniform(0.04, 0.2, 8)).astype(np.float32), 0.05)
    return csr(R), csr(Rh), lut, V


@pytest.mark.parametrize("iters,init_p", [(0, 0.5), (1, 0.5), (3, 0.5), (3, 0.1), (6, 0.3)])
def test_grad_matches_central_differences(iters, init_p):
    train, held, lut, V = _tiny_problem(11 + iters)
    ls = lut.log_sigma.astype(np.float64)
    w = 0.05
    loss, g_ls, g_w = oracle.grad(lut, ls, w, train, held, V, 0.5, init_p, iters)

    def f(theta):
        return oracle.grad(lut, theta[:-1], theta[-1], train, held, V, 0.5, init_p, iters, with_grad=False)

    theta = np.concatenate([ls, [w]])
    assert f(theta) == pytest.approx(loss, rel=1e-14)
    g = np.concatenate([g_ls, [g_w]])
    fd = np.array([_fd(f, theta, k) for k in range(len(theta))])
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max()), np.c_[g, fd]
    assert np.abs(g).max() > 0


def test_grad_loss_is_bp_then_heldout_loss():
    """The loss orc_grad reports is orc_bp's marginals fed to the held-out loss."""
    train, held, lut, V = _tiny_problem(5)
    ls = lut.log_sigma.astype(np.float64)
    w = float(np.float32(lut.outlier_w))   # the table's own (float) weight
    nu = oracle.nu_theta_edges(lut, ls, w, train["ray_off"], train["Z"], train["d"])
    nuh = oracle.nu_theta_edges(lut, ls, w, held["ray_off"], held["Z"], held["d"])
    _, _, p = oracle.bp(train["ray_off"], train["vox"], np.log(nu), V, 0.5, 0.1, math.log(w / 3.0), 4)
    ref = oracle.heldout_loss(held["ray_off"], held["vox"], nuh, w / 3.0, p)
    assert oracle.grad(lut, ls, w, train, held, V, 0.5, 0.1, 4, with_grad=False) == pytest.approx(ref, rel=1e-13)
    # and nu_theta_edges at the table's own values is the oracle's likelihood
    ln = oracle.log_nu_edges(lut, train["ray_off"], train["Z"], train["d"])
    assert np.allclose(np.log(nu), ln, rtol=0, atol=1e-12)
