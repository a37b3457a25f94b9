"""Seeded synthetic scenes, depth frames and noise tables.

The paper evaluates on a Gazebo scene, the augmented ICL-NUIM living room and
a RealSense D435 capture (Section IV); none of them is available here.  The
workloads below stand in for them with the same structure: indoor rooms with
boxes and spheres, 640x480-class depth images, 0.01-0.05 m voxels and a
Kinect-like depth noise whose standard deviation grows quadratically with
depth (Section III-F).  Every random draw comes from ``numpy.random.
default_rng(seed)`` with the seed fixed per workload, so every run sees the
same bytes.

Rendering is exact ray casting in FP64 against analytic primitives; the
z-depth of a pixel is the range to the first hit divided by the length of the
un-normalised pixel direction (a, b, 1).  Noise N(0, sigma_gen(z)) is then
added to z, 2% of pixels drop out to 0, and pixels that hit nothing are 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


# --------------------------------------------------------------------------
# plain records
# --------------------------------------------------------------------------
@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    res: float                      # voxel edge, metres
    origin: tuple = (0.0, 0.0, 0.0)  # min corner of voxel (0,0,0), metres

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def extent(self) -> np.ndarray:
        return np.array([self.nx, self.ny, self.nz], np.float64) * self.res

    @property
    def diagonal(self) -> float:
        return float(np.linalg.norm(self.extent))


@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    pose: np.ndarray  # (3, 4) float64 camera-to-world [R | c]; camera axes x right, y down, z forward


@dataclass
class NoiseTable:
    """Range-indexed sensor-noise table: log sigma at bin centres plus an outlier weight."""
    n_bins: int
    d_lo: float
    d_hi: float
    log_sigma: np.ndarray          # (n_bins,) float32
    outlier_w: float
    bias: Optional[np.ndarray] = None  # (n_bins,) float32 or None


@dataclass
class Frame:
    depth: np.ndarray  # (H, W) float32 z-depth in metres, 0 = invalid
    cam: Camera


@dataclass
class Workload:
    name: str
    grid: Grid
    prior: float
    frames: List[Frame]
    lut: NoiseTable
    iters: int
    heldout: List[Frame] = field(default_factory=list)
    description: str = ""
    init_p: float = 0.0   # first-pass message mu(o=1) on every edge; 0 selects the prior


def sigma_gen(z):
    """Generating depth-noise standard deviation (metres) as a function of z-depth."""
    z = np.asarray(z, np.float64)
    return 0.0012 + 0.0019 * (z - 0.4) ** 2


def noise_table(n_bins: int, d_hi: float, outlier_w: float = 0.02, d_lo: float = 0.0) -> NoiseTable:
    """log sigma_gen tabulated at bin centres d_lo + (k + 1/2) * (d_hi - d_lo) / n_bins."""
    delta = (d_hi - d_lo) / n_bins
    centres = d_lo + (np.arange(n_bins) + 0.5) * delta
    return NoiseTable(n_bins=n_bins, d_lo=float(d_lo), d_hi=float(d_hi),
                      log_sigma=np.log(sigma_gen(centres)).astype(np.float32),
                      outlier_w=float(outlier_w))


# --------------------------------------------------------------------------
# analytic primitives (all return the range t > 0 to the first hit, inf if none)
# --------------------------------------------------------------------------
class Prim:
    def hit(self, p: np.ndarray, d: np.ndarray) -> np.ndarray:  # p (3,), d (n,3) unit
        raise NotImplementedError

    def dist_to(self, q: np.ndarray) -> float:  # bounding-sphere clearance helper
        raise NotImplementedError


class Room(Prim):
    """Interior of an axis-aligned box seen from inside: distance to the walls."""

    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, np.float64)
        self.hi = np.asarray(hi, np.float64)

    def hit(self, p, d):
        with np.errstate(divide="ignore", invalid="ignore"):
            t_hi = (self.hi[None, :] - p[None, :]) / d
            t_lo = (self.lo[None, :] - p[None, :]) / d
        t = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
        return t.min(axis=1)


class Interior(Prim):
    """Interior of a union of overlapping axis-aligned boxes (rooms joined by openings), seen from
    inside: a ray leaving one box through a face that lies inside another box carries on in that one."""

    def __init__(self, boxes):
        self.boxes = [(np.asarray(lo, np.float64), np.asarray(hi, np.float64)) for lo, hi in boxes]

    def hit(self, p, d):
        t = np.zeros(d.shape[0])
        done = np.zeros(d.shape[0], bool)
        for _ in range(len(self.boxes) + 1):
            q = p[None, :] + (t + 1e-9)[:, None] * d
            nxt = t.copy()
            for lo, hi in self.boxes:
                inside = np.all((q > lo) & (q < hi), axis=1) & ~done
                if inside.any():
                    with np.errstate(divide="ignore", invalid="ignore"):
                        th = (hi[None, :] - q) / d
                        tl = (lo[None, :] - q) / d
                    ex = np.where(d > 0, th, np.where(d < 0, tl, np.inf)).min(axis=1)
                    nxt = np.where(inside, np.maximum(nxt, t + 1e-9 + ex), nxt)
            moved = nxt > t
            done |= ~moved
            t = nxt
            if done.all():
                break
        return np.where(t > 0, t, np.inf)


class Box(Prim):
    """Solid axis-aligned box seen from outside."""

    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, np.float64)
        self.hi = np.asarray(hi, np.float64)

    def hit(self, p, d):
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            ta = (self.lo[None, :] - p[None, :]) * inv
            tb = (self.hi[None, :] - p[None, :]) * inv
        ta = np.where(np.isnan(ta), -np.inf, ta)
        tb = np.where(np.isnan(tb), np.inf, tb)
        tn = np.minimum(ta, tb).max(axis=1)
        tf = np.maximum(ta, tb).min(axis=1)
        ok = (tn <= tf) & (tn > 0)
        return np.where(ok, tn, np.inf)

    @property
    def centre(self):
        return 0.5 * (self.lo + self.hi)

    @property
    def radius(self):
        return 0.5 * float(np.linalg.norm(self.hi - self.lo))


class Sphere(Prim):
    def __init__(self, c, r):
        self.c = np.asarray(c, np.float64)
        self.r = float(r)

    def hit(self, p, d):
        m = p - self.c
        b = d @ m
        cc = float(m @ m) - self.r * self.r
        disc = b * b - cc
        with np.errstate(invalid="ignore"):
            t = -b - np.sqrt(disc)
        return np.where((disc >= 0) & (t > 0), t, np.inf)

    @property
    def centre(self):
        return self.c

    @property
    def radius(self):
        return self.r


class FloorPlane(Prim):
    """Horizontal plane z = h seen from above."""

    def __init__(self, h):
        self.h = float(h)

    def hit(self, p, d):
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (self.h - p[2]) / d[:, 2]
        return np.where((d[:, 2] < 0) & (t > 0), t, np.inf)


# --------------------------------------------------------------------------
# cameras and rendering
# --------------------------------------------------------------------------
def look_at(c, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world pose [R | c] with camera z toward target, x right, y down."""
    c = np.asarray(c, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f], axis=1)
    return np.concatenate([R, c[:, None]], axis=1)


def render(cam: Camera, prims: List[Prim], cull: bool = False) -> np.ndarray:
    """Exact FP64 z-depth image (inf where nothing is hit).  With cull, a bounded primitive is only
    intersected with the rays that meet its bounding sphere (slightly enlarged) before their current
    nearest hit; the others cannot change."""
    u, v = np.meshgrid(np.arange(cam.W, dtype=np.float64), np.arange(cam.H, dtype=np.float64))
    a = ((u - cam.cx) / cam.fx).ravel()
    b = ((v - cam.cy) / cam.fy).ravel()
    dirc = np.stack([a, b, np.ones_like(a)], axis=1)
    ln = np.linalg.norm(dirc, axis=1)
    R = cam.pose[:, :3]
    p = cam.pose[:, 3].copy()
    dw = (dirc @ R.T) / ln[:, None]
    t = np.full(a.shape, np.inf)
    for pr in prims:
        if cull and isinstance(pr, (Box, Sphere)):
            m = p - pr.centre
            r = pr.radius * 1.001 + 1e-6
            b = dw @ m
            disc = b * b - (float(m @ m) - r * r)
            sq = np.sqrt(np.maximum(disc, 0.0))
            cand = np.nonzero((disc >= 0) & (sq - b > 0) & (-b - sq < t))[0]
            if cand.size:
                t[cand] = np.minimum(t[cand], pr.hit(p, dw[cand]))
        else:
            np.minimum(t, pr.hit(p, dw), out=t)
    return (t / ln).reshape(cam.H, cam.W)


def noisy_depth(z: np.ndarray, rng: np.random.Generator, dropout: float = 0.02) -> np.ndarray:
    """Add N(0, sigma_gen(z)) to z, drop out a fraction of pixels, mark misses as 0."""
    valid = np.isfinite(z)
    zz = np.where(valid, z, 1.0)
    noise = rng.standard_normal(z.shape) * sigma_gen(zz)
    out = np.where(valid, zz + noise, 0.0)
    drop = rng.random(z.shape) < dropout
    out = np.where(drop, 0.0, out)
    out = np.where(out > 0, out, 0.0)
    return out.astype(np.float32)


# --------------------------------------------------------------------------
# scene builders
# --------------------------------------------------------------------------
def _room_primitives(rng, room_lo, room_hi, n_prims, ring_c, ring_r, ring_h, clearance=0.3):
    """Random boxes and spheres inside a room, kept `clearance` away from the camera ring."""
    prims: List[Prim] = []
    lo = np.asarray(room_lo, np.float64)
    hi = np.asarray(room_hi, np.float64)
    tries = 0
    while len(prims) < n_prims:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place primitives")
        if rng.random() < 0.5:
            size = rng.uniform(0.2, 0.8, 3)
            on_floor = rng.random() < 0.6
            xy = rng.uniform(lo[:2] + size[:2] / 2, hi[:2] - size[:2] / 2)
            z0 = lo[2] if on_floor else rng.uniform(lo[2], hi[2] - size[2])
            blo = np.array([xy[0] - size[0] / 2, xy[1] - size[1] / 2, z0])
            pr: Prim = Box(blo, blo + size)
        else:
            r = rng.uniform(0.1, 0.4)
            c = rng.uniform(lo + r, hi - r)
            if rng.random() < 0.6:
                c[2] = lo[2] + r
            pr = Sphere(c, r)
        q = pr.centre
        rho = math.hypot(q[0] - ring_c[0], q[1] - ring_c[1])
        dist_ring = math.hypot(rho - ring_r, q[2] - ring_h)
        if dist_ring - pr.radius > clearance:
            prims.append(pr)
    return prims


def _ring_cameras(rng, n, centre, radius, height, W, H, f, cx, cy):
    phase = rng.uniform(0, 2 * math.pi)
    cams = []
    for k in range(n):
        phi = phase + 2 * math.pi * k / n
        c = (centre[0] + radius * math.cos(phi), centre[1] + radius * math.sin(phi), height)
        cams.append(Camera(W, H, f, f, cx, cy, look_at(c, (centre[0], centre[1], height))))
    return cams


def make_plain_64x48(seed: int = 1) -> Workload:
    """One 64x48 frame over a 1.6 m scene: floor, 0.4 m box, 0.3 m sphere; 32^3 at 0.05 m."""
    rng = np.random.default_rng(seed)
    grid = Grid(32, 32, 32, 0.05, (0.0, 0.0, 0.0))
    floor_h = 0.1
    while True:
        bxy = rng.uniform(0.25, 0.95, 2)
        sxy = rng.uniform(0.35, 1.25, 2)
        if np.linalg.norm((bxy + 0.2) - sxy) > 0.6:
            break
    box = Box([bxy[0], bxy[1], floor_h], [bxy[0] + 0.4, bxy[1] + 0.4, floor_h + 0.4])
    sph = Sphere([sxy[0], sxy[1], floor_h + 0.3], 0.3)
    target = np.array([0.8, 0.8, 0.3])
    az = rng.uniform(0, 2 * math.pi)
    el = math.radians(rng.uniform(55, 62))
    dist = rng.uniform(0.9, 1.1)
    c = target + dist * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    cam = Camera(64, 48, 60.0, 60.0, 32.0, 24.0, look_at(c, target))
    z = render(cam, [FloorPlane(floor_h), box, sph])
    depth = noisy_depth(z, rng)
    lut = noise_table(32, grid.diagonal)
    return Workload("plain_64x48", grid, 0.5, [Frame(depth, cam)], lut, 10,
                    description="1 frame 64x48 (f=60), 32^3 grid @0.05 m, 32-bin LUT, w=0.02, 10 iters")


def _room_workload(name, seed, n, res, n_frames, W, H, f, n_prims, n_bins, iters, heldout_idx=(),
                   description="", init_p=0.0):
    rng = np.random.default_rng(seed)
    grid = Grid(n, n, n, res, (0.0, 0.0, 0.0))
    ext = n * res
    inset = 2 * res
    room_lo = np.array([inset, inset, inset])
    room_hi = np.array([ext - inset] * 3)
    centre = (ext / 2, ext / 2)
    ring_r, ring_h = 1.5, 1.2
    prims = _room_primitives(rng, room_lo, room_hi, n_prims, centre, ring_r, ring_h)
    scene: List[Prim] = [Room(room_lo, room_hi)] + prims
    cams = _ring_cameras(rng, n_frames + len(heldout_idx), centre, ring_r, ring_h, W, H, f, W / 2, H / 2)
    frames, held = [], []
    for k, cam in enumerate(cams):
        fr = Frame(noisy_depth(render(cam, scene), rng), cam)
        (held if k in heldout_idx else frames).append(fr)
    lut = noise_table(n_bins, grid.diagonal)
    return Workload(name, grid, 0.5, frames, lut, iters, held, description, init_p)


def make_room_30x640x480(seed: int = 2) -> Workload:
    """30 frames 640x480 (f=525) on a 1.5 m camera ring in a 5.12 m room; 256^3 @0.02 m."""
    # Rays cross 200-480 voxels here; with every first-pass message at the
    # non-informative prior 0.5 the visibility 0.5^i vanishes long before the
    # surface and BP stays at the all-zero fixed point.  Section IV-A
    # initialises the occupancy variables at 0.1 for exactly this reason.
    return _room_workload("room_30x640x480", seed, 256, 0.02, 30, 640, 480, 525.0, 20, 64, 20,
                          description="30 frames 640x480 (f=525) ring r=1.5 m h=1.2 m, 20 primitives, "
                                      "256^3 grid @0.02 m, 64-bin LUT, w=0.02, first pass 0.1, 20 iters",
                          init_p=0.1)


def make_room_small(seed: int = 5, n: int = 64, res: float = 0.08, n_frames: int = 4,
                    W: int = 80, H: int = 60, iters: int = 10) -> Workload:
    """Reduced room (same generator) for parity tests that the oracle finishes in seconds."""
    f = 525.0 * W / 640.0
    return _room_workload(f"room_{n_frames}x{W}x{H}_{n}^3", seed, n, res, n_frames, W, H, f, 6, 64, iters,
                          description=f"{n_frames} frames {W}x{H} (f={f}), {n}^3 grid @{res} m, 64-bin LUT")


def make_diff_8x160x120(seed: int = 4) -> Workload:
    """8 training + 2 held-out frames 160x120 (f=131.25) over a 128^3 grid @0.04 m; first pass 0.1
    (Section IV-A) as for the 256^3 room, whose rays are as long in voxels."""
    return _room_workload("diff_8x160x120", seed, 128, 0.04, 8, 160, 120, 131.25, 10, 64, 10,
                          heldout_idx=(3, 7),
                          description="8 frames 160x120 (f=131.25) + 2 held-out, 128^3 @0.04 m, first pass 0.1, "
                                      "10 iters", init_p=0.1)


def make_diff_small(seed: int = 6) -> Workload:
    """Reduced differentiation case (same generator) the oracle's finite differences finish in seconds:
    4 training + 2 held-out frames 40x30 over a 32^3 grid @0.16 m, 6 passes, first pass 0.1."""
    return _room_workload("diff_small", seed, 32, 0.16, 4, 40, 30, 32.8125, 6, 16, 6, heldout_idx=(1, 4),
                          description="4 frames 40x30 + 2 held-out, 32^3 @0.16 m, 16-bin LUT, first pass 0.1, "
                                      "6 iters", init_p=0.1)


def make_corridor_60x424x240(seed: int = 9) -> Workload:
    """A 10 m camera path along a corridor that opens into a room, 60 keyframes of 424x240 depth
    (f = 212, c = (212, 120)), 200 seeded boxes and spheres, 512x512x256 grid at 0.02 m (10.24 x 10.24 x
    5.12 m), 64-bin table, first pass 0.1, 30 passes.

    Corridor: x 0.1-6.1 m, y 4.0-6.2 m, z 0.1-2.8 m; room: x 6.0-10.14 m, y 0.1-10.14 m, z 0.1-3.6 m.
    The path runs 5.4 m down the corridor's centre line at 1.3 m, then 4.6 m along a right-hand arc of
    radius 2.5 m in the room; each camera looks along the path, 8 degrees down, turned by up to
    +-25 degrees (seeded).  Primitives stand on the floor or float, kept 0.35 m from the path."""
    rng = np.random.default_rng(seed)
    res = 0.02
    grid = Grid(512, 512, 256, res, (0.0, 0.0, 0.0))
    corr = (np.array([0.1, 4.0, 0.1]), np.array([6.1, 6.2, 2.8]))
    room = (np.array([6.0, 0.1, 0.1]), np.array([10.14, 10.14, 3.6]))
    h_cam, L1, R = 1.3, 5.4, 2.5

    def path(s):
        if s <= L1:
            return np.array([0.6 + s, 5.1, h_cam]), np.array([1.0, 0.0, 0.0])
        a = (s - L1) / R
        return (np.array([0.6 + L1 + R * math.sin(a), 5.1 - R + R * math.cos(a), h_cam]),
                np.array([math.cos(a), -math.sin(a), 0.0]))

    samples = np.array([path(s)[0] for s in np.linspace(0.0, 10.0, 201)])
    prims: List[Prim] = []
    tries = 0
    while len(prims) < 200:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place primitives")
        lo, hi = corr if rng.random() < 0.3 else room
        if rng.random() < 0.5:
            size = rng.uniform(0.1, 0.6, 3)
            xy = rng.uniform(lo[:2] + size[:2] / 2, hi[:2] - size[:2] / 2)
            z0 = lo[2] if rng.random() < 0.6 else rng.uniform(lo[2], hi[2] - size[2])
            blo = np.array([xy[0] - size[0] / 2, xy[1] - size[1] / 2, z0])
            pr: Prim = Box(blo, blo + size)
        else:
            r = rng.uniform(0.05, 0.3)
            c = rng.uniform(lo + r, hi - r)
            if rng.random() < 0.6:
                c[2] = lo[2] + r
            pr = Sphere(c, r)
        if np.min(np.linalg.norm(samples - pr.centre[None, :], axis=1)) - pr.radius > 0.35:
            prims.append(pr)
    scene: List[Prim] = [Interior([corr, room])] + prims
    frames = []
    for k in range(60):
        c, fwd = path(10.0 * k / 59)
        yaw = math.radians(rng.uniform(-25.0, 25.0))
        pitch = math.radians(-8.0)
        cy, sy = math.cos(yaw), math.sin(yaw)
        f2 = np.array([cy * fwd[0] - sy * fwd[1], sy * fwd[0] + cy * fwd[1], 0.0])
        look = np.array([f2[0] * math.cos(pitch), f2[1] * math.cos(pitch), math.sin(pitch)])
        cam = Camera(424, 240, 212.0, 212.0, 212.0, 120.0, look_at(c, c + look))
        frames.append(Frame(noisy_depth(render(cam, scene, cull=True), rng), cam))
    return Workload("corridor_60x424x240", grid, 0.5, frames, noise_table(64, grid.diagonal), 30, [],
                    "60 frames 424x240 (f=212) along a 10 m corridor-and-room path, 200 primitives, "
                    "512x512x256 grid @0.02 m, 64-bin LUT, w=0.02, first pass 0.1, 30 iters", 0.1)


BATCH64_SCENES = 64


def batch_scene_size(index: int, seed: int = 7):
    """(grid edge in voxels, frame count) of scene `index` of the 64-scene batch, without rendering it:
    the first two draws of make_batch_scene."""
    rng = np.random.default_rng([seed, index])
    n = 8 * int(rng.integers(8, 25))
    return n, int(rng.integers(8, 61))


def make_batch_scene(index: int, seed: int = 7) -> Workload:
    """Scene `index` of the 64-scene batch: a room whose grid edge is uniform in 64..192 voxels at
    0.03 m, 4-15 primitives, 8-60 frames of 320x240 (f = 262.5, c = (160, 120)) on a camera ring at
    0.28 / 0.23 of the room size, 64-bin table, first pass 0.1, 15 passes."""
    rng = np.random.default_rng([seed, index])
    n = 8 * int(rng.integers(8, 25))
    res = 0.03
    n_frames = int(rng.integers(8, 61))
    ext = n * res
    grid = Grid(n, n, n, res, (0.0, 0.0, 0.0))
    inset = 2 * res
    room_lo = np.array([inset] * 3)
    room_hi = np.array([ext - inset] * 3)
    centre = (ext / 2, ext / 2)
    ring_r, ring_h = 0.28 * ext, 0.23 * ext
    prims = _room_primitives(rng, room_lo, room_hi, int(rng.integers(4, 16)), centre, ring_r, ring_h,
                             clearance=0.08 * ext)
    scene: List[Prim] = [Room(room_lo, room_hi)] + prims
    cams = _ring_cameras(rng, n_frames, centre, ring_r, ring_h, 320, 240, 262.5, 160.0, 120.0)
    frames = [Frame(noisy_depth(render(cam, scene), rng), cam) for cam in cams]
    return Workload(f"batch64_{index}", grid, 0.5, frames, noise_table(64, grid.diagonal), 15, [],
                    f"{n}^3 @0.03 m, {n_frames} frames 320x240, first pass 0.1, 15 iters", 0.1)


def make_batch_small(seed: int = 8) -> List[Workload]:
    """Three small rooms of different sizes (the room generator) for batched-context parity tests."""
    return [make_room_small(seed=seed + k, n=n, res=0.08, n_frames=3, W=64, H=48, iters=8)
            for k, n in enumerate((64, 56, 48))]


def theta_off(lut: NoiseTable, factor: float = 1.3) -> NoiseTable:
    """The noise table a fit starts from: every sigma and the outlier weight scaled by `factor`."""
    return NoiseTable(lut.n_bins, lut.d_lo, lut.d_hi,
                      (np.asarray(lut.log_sigma, np.float64) + np.log(factor)).astype(np.float32),
                      float(np.float32(lut.outlier_w * factor)), lut.bias)


WORKLOADS: Dict[str, Callable[..., Workload]] = {
    "plain_64x48": make_plain_64x48,
    "diff_small": make_diff_small,
    "room_30x640x480": make_room_30x640x480,
    "room_small": make_room_small,
    "diff_8x160x120": make_diff_8x160x120,
    "corridor_60x424x240": make_corridor_60x424x240,
}


def make_workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
