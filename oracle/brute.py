"""Literal, exponential-cost evaluations of the paper's definitions.

TEST INFRASTRUCTURE ONLY.  These routines pin the FP64 oracle: they share no
formula with it.  Each one enumerates what a definition says instead of using
the paper's O(N) simplifications.

* ``psi_sum`` -- Eq. "depth_potential" (and its case form): psi_r(o, d) is
  nu(d_i) when d is the depth of the first occupied voxel i, else 0.  The depth
  variable's incoming message is uniform (Section III-C, "Depth Variable to Ray
  Depth Potential Messages"), so summing psi over d leaves nu of the first
  occupied voxel.  For the all-empty configuration the value is nu_bg (a
  reading; nu_bg = 0 is the literal paper).
* ``factor_to_node`` -- Eq. "factor_to_node" for one ray factor: sum over
  every configuration of the other voxels (2^(N-1) terms per target).
* ``tree_marginals`` -- exact marginals of p(o) proportional to
  prod_i phi_i(o_i) * sum_d psi(o, d) for one ray (Eq. 1 restricted to one
  ray, with the prior factor of Eq. "prior_potential").
* ``loopy_bp`` -- generic flooding sum-product on an explicit factor graph of
  several rays (Eqs. "node_to_factor", "factor_to_node", and the marginal
  equation), with 2-vector messages (no log-odds bookkeeping).
* ``march_cells`` / ``segment_lengths`` -- voxels crossed by a segment, found
  by fine-step marching and by exact slab clipping in FP64.

Every function accepts floats; ``factor_to_node_exact`` and
``tree_marginals_exact`` use Python ``fractions.Fraction`` for exact values.
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from typing import Dict, List, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------
# one ray factor
# --------------------------------------------------------------------------
def _configs(N: int) -> np.ndarray:
    return ((np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1).astype(np.int8)


def psi_sum(o: Sequence[int], nu: Sequence, nu_bg):
    """sum over the depth variable of psi_r(o, d), with psi as Eq. "depth_potential".

    The depth the potential accepts is d_r = sum_i o_i prod_{j<i} (1 - o_j) d_i,
    i.e. the depth of the first occupied voxel; only that value of d gives a
    non-zero term, equal to nu(d_i).  No occupied voxel: the background term.
    """
    total = 0
    for d_index in range(len(nu) + 1):           # d ranges over d_1..d_N and "none"
        for i in range(len(nu)):
            first = o[i] == 1 and all(o[j] == 0 for j in range(i))
            if first and d_index == i:
                total = total + nu[i]
        if d_index == len(nu) and all(x == 0 for x in o):
            total = total + nu_bg
    return total


def factor_to_node(m1: Sequence[float], nu: Sequence[float], nu_bg: float) -> np.ndarray:
    """Ray factor -> occupancy messages by enumeration; returns log-odds lambda_i.

    m1[j] = mu_{o_j -> psi}(o_j = 1), normalised so mu(o_j=0) = 1 - m1[j].
    """
    m1 = np.asarray(m1, np.float64)
    nu = np.asarray(nu, np.float64)
    N = len(m1)
    cf = _configs(N)
    # sum_d psi(o, d): first occupied index via the product rule of the equation
    first_mask = np.zeros((2 ** N, N), bool)
    none_before = np.ones(2 ** N, bool)
    for i in range(N):
        first_mask[:, i] = (cf[:, i] == 1) & none_before
        none_before &= cf[:, i] == 0
    ps = (first_mask * nu[None, :]).sum(axis=1) + np.where(none_before, nu_bg, 0.0)
    M = np.where(cf == 1, m1[None, :], 1.0 - m1[None, :])
    lam = np.zeros(N)
    for i in range(N):
        Mi = M.copy()
        Mi[:, i] = 1.0
        w = ps * Mi.prod(axis=1)
        mu1 = w[cf[:, i] == 1].sum()
        mu0 = w[cf[:, i] == 0].sum()
        lam[i] = np.log(mu1) - np.log(mu0)
    return lam


def factor_to_node_exact(m1: Sequence[Fraction], nu: Sequence[Fraction], nu_bg: Fraction
                         ) -> List[Tuple[Fraction, Fraction]]:
    """Exact (mu(o_i=1), mu(o_i=0)) pairs by enumeration in rational arithmetic."""
    N = len(m1)
    out = []
    for i in range(N):
        mu = [Fraction(0), Fraction(0)]
        for o in itertools.product((0, 1), repeat=N):
            w = psi_sum(o, nu, nu_bg)
            for j in range(N):
                if j != i:
                    w *= m1[j] if o[j] == 1 else (1 - m1[j])
            mu[o[i]] += w
        out.append((mu[1], mu[0]))
    return out


def tree_marginals(prior: float, nu: Sequence[float], nu_bg: float) -> np.ndarray:
    """Exact p(o_i = 1) for one ray and its voxels' priors (a tree)."""
    nu = np.asarray(nu, np.float64)
    N = len(nu)
    cf = _configs(N)
    first_mask = np.zeros((2 ** N, N), bool)
    none_before = np.ones(2 ** N, bool)
    for i in range(N):
        first_mask[:, i] = (cf[:, i] == 1) & none_before
        none_before &= cf[:, i] == 0
    ps = (first_mask * nu[None, :]).sum(axis=1) + np.where(none_before, nu_bg, 0.0)
    phi = np.where(cf == 1, prior, 1.0 - prior).prod(axis=1)
    w = phi * ps
    return (w[:, None] * cf).sum(axis=0) / w.sum()


def tree_marginals_exact(prior: Fraction, nu: Sequence[Fraction], nu_bg: Fraction) -> List[Fraction]:
    N = len(nu)
    num = [Fraction(0)] * N
    Z = Fraction(0)
    for o in itertools.product((0, 1), repeat=N):
        w = psi_sum(o, nu, nu_bg)
        for x in o:
            w *= prior if x == 1 else (1 - prior)
        Z += w
        for i in range(N):
            if o[i]:
                num[i] += w
    return [n / Z for n in num]


# --------------------------------------------------------------------------
# generic loopy BP on an explicit factor graph
# --------------------------------------------------------------------------
def loopy_bp(rays: List[List[int]], nus: List[Sequence[float]], nu_bg: float, V: int,
             prior: float, init_p: float, iters: int) -> np.ndarray:
    """Flooding sum-product; returns p(o_v = 1) for v in 0..V-1.

    Factors: a prior phi_v per voxel and one ray factor per ray (its depth
    variable summed out under a uniform message).  Iteration 1 sends the
    Bernoulli(init_p) message from every voxel to every ray factor; later
    iterations send phi_v times the other rays' messages (Eq. "node_to_factor").
    Every ray factor then answers by enumeration (Eq. "factor_to_node").
    """
    for r in rays:
        assert len(set(r)) == len(r), "a ray visits each voxel once"
    phi = np.array([1.0 - prior, prior])
    # factor -> variable messages, as normalised 2-vectors per (ray, position)
    f2v = [[np.array([0.5, 0.5]) for _ in r] for r in rays]
    for it in range(iters):
        v2f = []
        for ri, r in enumerate(rays):
            msgs = []
            for pi, v in enumerate(r):
                if it == 0:
                    m = np.array([1.0 - init_p, init_p])
                else:
                    m = phi.copy()
                    for rj, r2 in enumerate(rays):
                        for pj, v2 in enumerate(r2):
                            if v2 == v and rj != ri:
                                m = m * f2v[rj][pj]
                    m = m / m.sum()
                msgs.append(m)
            v2f.append(msgs)
        new = []
        for ri, r in enumerate(rays):
            m1 = [v2f[ri][pi][1] for pi in range(len(r))]
            lam = factor_to_node(m1, nus[ri], nu_bg)
            pr1 = 1.0 / (1.0 + np.exp(-lam))
            new.append([np.array([1.0 - q, q]) for q in pr1])
        f2v = new
    p = np.zeros(V)
    for v in range(V):
        b = phi.copy()
        for ri, r in enumerate(rays):
            for pi, v2 in enumerate(r):
                if v2 == v:
                    b = b * f2v[ri][pi]
        p[v] = b[1] / b.sum()
    return p


# --------------------------------------------------------------------------
# traversal references
# --------------------------------------------------------------------------
def march_cells(o, k, t0: float, t1: float, n, step: float = 1e-5) -> List[Tuple[int, int, int]]:
    """Cells visited by points o + t k, t in [t0, t1], sampled every `step` voxel of path."""
    o = np.asarray(o, np.float64)
    k = np.asarray(k, np.float64)
    speed = float(np.linalg.norm(k))           # voxels per unit t
    n_s = max(2, int(np.ceil((t1 - t0) * speed / step)) + 1)
    t = np.linspace(t0, t1, n_s)
    pts = o[None, :] + t[:, None] * k[None, :]
    c = np.floor(pts).astype(np.int64)
    for q in range(3):
        c[:, q] = np.clip(c[:, q], 0, int(n[q]) - 1)
    keep = np.ones(len(c), bool)
    keep[1:] = np.any(c[1:] != c[:-1], axis=1)
    return [tuple(int(x) for x in row) for row in c[keep]]


def segment_lengths(o, k, t0: float, t1: float, n) -> Dict[Tuple[int, int, int], float]:
    """Exact FP64 length (in voxel units) of the segment inside every voxel it meets."""
    o = np.asarray(o, np.float64)
    k = np.asarray(k, np.float64)
    speed = float(np.linalg.norm(k))
    lo = np.minimum(o + t0 * k, o + t1 * k)
    hi = np.maximum(o + t0 * k, o + t1 * k)
    rng = [range(max(0, int(np.floor(lo[q])) - 1), min(int(n[q]), int(np.floor(hi[q])) + 2)) for q in range(3)]
    out = {}
    for x in rng[0]:
        for y in rng[1]:
            for z in rng[2]:
                a, b = t0, t1
                cell = (x, y, z)
                for q in range(3):
                    if k[q] == 0.0:
                        if not (cell[q] <= o[q] < cell[q] + 1):
                            a, b = 1.0, 0.0
                        continue
                    ta = (cell[q] - o[q]) / k[q]
                    tb = (cell[q] + 1 - o[q]) / k[q]
                    a = max(a, min(ta, tb))
                    b = min(b, max(ta, tb))
                if b >= a:
                    out[cell] = (b - a) * speed
    return out


def segments(o, k, t0: float, t1: float, n) -> List[Tuple[Tuple[int, int, int], float, float]]:
    """Every voxel the segment o + t k, t in [t0, t1], meets, with its exact FP64 entry and exit t (slab
    clipping), in order of entry; voxels touched at a single point are left out."""
    o = np.asarray(o, np.float64)
    k = np.asarray(k, np.float64)
    lo = np.minimum(o + t0 * k, o + t1 * k)
    hi = np.maximum(o + t0 * k, o + t1 * k)
    rng = [range(max(0, int(np.floor(lo[q])) - 1), min(int(n[q]), int(np.floor(hi[q])) + 2)) for q in range(3)]
    out = []
    for x in rng[0]:
        for y in rng[1]:
            for z in rng[2]:
                a, b = t0, t1
                cell = (x, y, z)
                for q in range(3):
                    if k[q] == 0.0:
                        if not (cell[q] <= o[q] < cell[q] + 1):
                            a, b = 1.0, 0.0
                        continue
                    ta = (cell[q] - o[q]) / k[q]
                    tb = (cell[q] + 1 - o[q]) / k[q]
                    a = max(a, min(ta, tb))
                    b = min(b, max(ta, tb))
                if b > a:
                    out.append((cell, a, b))
    return sorted(out, key=lambda c: c[1])
