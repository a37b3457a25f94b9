"""FP64 CPU oracle for ray-MRF loopy belief propagation (MRFMap, arXiv 2006.03512).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline and reference legs are its only users; the product path
never imports it.  It shares no code with the CUDA library.

``mrf_oracle.c`` holds the arithmetic (traversal recipe, sensor likelihood,
ray messages of Eqs. "pos"/"neg", flooding BP); ``brute.py`` holds literal
enumerations of the paper's definitions (Eq. "factor_to_node" over all 2^N
occupancy configurations, generic sum-product on an explicit factor graph)
that pin it.  This module compiles the C file with gcc and wraps it with
ctypes and numpy.

Parity pins, per function (see tests/test_oracle_pins.py):
  ray_messages          2^N enumeration of Eq. "factor_to_node"; closed forms
  ray_messages_divfree  agrees with ray_messages; enumeration
  bp                    exact tree marginals (one ray); generic loopy BP
  traversal             fine-step FP64 marching; exact slab intersection
  log_nu                Gaussian normalisation; table interpolation nodes
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fno-strict-aliasing", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("res", C.c_float),
                ("origin", C.c_float * 3)]


class _Camera(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("pose", C.c_double * 12)]


class _Lut(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("d_lo", C.c_float), ("d_hi", C.c_float),
                ("log_sigma", C.c_void_p), ("outlier_w", C.c_float), ("bias", C.c_void_p)]


class _Ray(C.Structure):
    _fields_ = [("o", C.c_float * 3), ("k", C.c_float * 3), ("inv", C.c_float * 3),
                ("t0", C.c_float), ("t1", C.c_float), ("Z", C.c_float),
                ("s", C.c_int32 * 3), ("e", C.c_int32 * 3), ("N", C.c_int32)]


RAY_DTYPE = np.dtype([("o", "<f4", 3), ("k", "<f4", 3), ("inv", "<f4", 3), ("t0", "<f4"),
                      ("t1", "<f4"), ("Z", "<f4"), ("s", "<i4", 3), ("e", "<i4", 3), ("N", "<i4")])
assert RAY_DTYPE.itemsize == C.sizeof(_Ray)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_frame_setup.argtypes = [P, P, P, P, P]
            L.orc_frame_walk.argtypes = [P, C.c_int64, P, P, P, P]
            L.orc_log_nu.argtypes = [P, C.c_double, C.c_double]
            L.orc_log_nu.restype = C.c_double
            L.orc_log_sigma_at.argtypes = [P, C.c_double]
            L.orc_log_sigma_at.restype = C.c_double
            L.orc_log_nu_edges.argtypes = [P, C.c_int64, P, P, P, P]
            L.orc_default_log_nu_bg.argtypes = [P]
            L.orc_default_log_nu_bg.restype = C.c_double
            L.orc_ray_messages.argtypes = [C.c_int, P, P, C.c_double, P, P]
            L.orc_ray_messages_divfree.argtypes = [C.c_int, P, P, C.c_double, P]
            L.orc_transpose.argtypes = [C.c_int64, P, C.c_int64, P, P]
            L.orc_bp.argtypes = [C.c_int64, P, P, P, C.c_int64, C.c_double, C.c_double, C.c_double,
                                 C.c_int, P, P, P]
            L.orc_bp.restype = C.c_int
            L.orc_nu_theta_edges.argtypes = [P, P, C.c_double, C.c_int64, P, P, P, P]
            L.orc_heldout_loss.argtypes = [C.c_int64, P, P, P, C.c_double, P, P, P, P]
            L.orc_heldout_loss.restype = C.c_double
            L.orc_ray_messages_adjoint.argtypes = [C.c_int, P, P, C.c_double, P, P, P, P, P]
            L.orc_grad.argtypes = [P, P, C.c_double, C.c_int64, P, P, P, P, C.c_int64, P, P, P, P, C.c_int64,
                                   C.c_double, C.c_double, C.c_int, P, P, P]
            L.orc_grad.restype = C.c_int
            L.orc_omega_ray.argtypes = [C.c_int, P, P, P, P, C.c_double, C.c_float, P]
            L.orc_omega_ray.restype = C.c_int
            L.orc_omega_frame.argtypes = [P, P, P, P, P, P]
            L.orc_omega_frame.restype = C.c_int64
            L.orc_bp_variants.argtypes = [C.c_int64, P, P, P, C.c_int64, C.c_double, C.c_double, C.c_double,
                                          C.c_int, P, P, P, P, P]
            L.orc_bp_variants.restype = C.c_int
            L.orc_frame_walk_seg.argtypes = [P, C.c_int64, P, P, P, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# --------------------------------------------------------------------------
# struct marshalling (inputs come from the synth package's plain records)
# --------------------------------------------------------------------------
class _LutHold:
    def __init__(self, lut):
        self.ls = np.ascontiguousarray(lut.log_sigma, np.float32)
        self.bias = None if lut.bias is None else np.ascontiguousarray(lut.bias, np.float32)
        self.s = _Lut(int(lut.n_bins), float(lut.d_lo), float(lut.d_hi), self.ls.ctypes.data,
                      float(lut.outlier_w), 0 if self.bias is None else self.bias.ctypes.data)


def _grid(g) -> _Grid:
    return _Grid(int(g.nx), int(g.ny), int(g.nz), float(g.res), (C.c_float * 3)(*[float(x) for x in g.origin]))


def _cam(c) -> _Camera:
    pose = np.asarray(c.pose, np.float64).reshape(12)
    return _Camera(int(c.W), int(c.H), float(c.fx), float(c.fy), float(c.cx), float(c.cy),
                   (C.c_double * 12)(*pose.tolist()))


# --------------------------------------------------------------------------
# traversal
# --------------------------------------------------------------------------
def frame_setup(grid, cam, depth, lut) -> np.ndarray:
    """Per-pixel ray set-up (structured array with o, k, inv, t0, t1, Z, s, e, N)."""
    depth = np.ascontiguousarray(depth, np.float32)
    assert depth.shape == (cam.H, cam.W)
    rays = np.zeros(cam.W * cam.H, RAY_DTYPE)
    g, c, lh = _grid(grid), _cam(cam), _LutHold(lut)
    lib().orc_frame_setup(C.byref(g), C.byref(c), C.byref(lh.s), _p(depth), _p(rays))
    return rays


def frame_walk(grid, rays: np.ndarray):
    """Walk rays into a CSR: (ray_off int64[R+1], vox uint32[E], d float32[E])."""
    N = rays["N"].astype(np.int64)
    ray_off = np.zeros(len(rays) + 1, np.int64)
    np.cumsum(N, out=ray_off[1:])
    E = int(ray_off[-1])
    vox = np.zeros(max(E, 1), np.uint32)
    d = np.zeros(max(E, 1), np.float32)
    g = _grid(grid)
    rays = np.ascontiguousarray(rays)
    lib().orc_frame_walk(C.byref(g), len(rays), _p(rays), _p(ray_off), _p(vox), _p(d))
    return ray_off, vox[:E], d[:E]


def frame_walk_seg(grid, rays: np.ndarray, ray_off: np.ndarray):
    """The walk with each voxel's entry and exit range: (vox, d, t_in, t_out)."""
    E = int(ray_off[-1])
    out = [np.zeros(max(E, 1), t) for t in (np.uint32, np.float32, np.float32, np.float32)]
    g = _grid(grid)
    rays = np.ascontiguousarray(rays)
    lib().orc_frame_walk_seg(C.byref(g), len(rays), _p(rays), _p(np.ascontiguousarray(ray_off, np.int64)),
                             *[_p(a) for a in out])
    return [a[:E] for a in out]


def length_weights(grid, frames, lut) -> np.ndarray:
    """w_e = min(1, l_e / h) per edge of trace_frames(grid, frames, lut), l_e the traversed length."""
    ws = []
    for fr in frames:
        rays = frame_setup(grid, fr.cam, fr.depth, lut)
        N = rays["N"].astype(np.int64)
        ro = np.zeros(len(rays) + 1, np.int64)
        np.cumsum(N, out=ro[1:])
        _, _, ti, to = frame_walk_seg(grid, rays, ro)
        ws.append(np.minimum(1.0, (to.astype(np.float64) - ti.astype(np.float64)) / float(np.float32(grid.res))))
    return np.concatenate(ws) if ws else np.zeros(0)


def trace_frame(grid, cam, depth, lut):
    """Set-up + walk for one frame: dict(ray_off, vox, d, Z, N, rays)."""
    rays = frame_setup(grid, cam, depth, lut)
    ray_off, vox, d = frame_walk(grid, rays)
    return dict(ray_off=ray_off, vox=vox, d=d, Z=rays["Z"].copy(), N=rays["N"].copy(), rays=rays)


def log_nu(lut, d: float, Z: float) -> float:
    lh = _LutHold(lut)
    return float(lib().orc_log_nu(C.byref(lh.s), float(d), float(Z)))


def log_sigma_at(lut, d: float) -> float:
    lh = _LutHold(lut)
    return float(lib().orc_log_sigma_at(C.byref(lh.s), float(d)))


def log_nu_edges(lut, ray_off, Z, d) -> np.ndarray:
    ray_off = np.ascontiguousarray(ray_off, np.int64)
    Z = np.ascontiguousarray(Z, np.float32)
    d = np.ascontiguousarray(d, np.float32)
    out = np.zeros(max(len(d), 1), np.float64)
    lh = _LutHold(lut)
    lib().orc_log_nu_edges(C.byref(lh.s), len(ray_off) - 1, _p(ray_off), _p(Z), _p(d), _p(out))
    return out[:len(d)]


def default_log_nu_bg(lut) -> float:
    """log of the uniform outlier density w / d_hi (-inf when w = 0), from the table's float fields."""
    lh = _LutHold(lut)
    return float(lib().orc_default_log_nu_bg(C.byref(lh.s)))


# --------------------------------------------------------------------------
# messages and inference
# --------------------------------------------------------------------------
def ray_messages(L, log_nu_v, log_nu_bg: float) -> np.ndarray:
    L = np.ascontiguousarray(L, np.float64)
    ln = np.ascontiguousarray(log_nu_v, np.float64)
    N = len(L)
    out = np.zeros(N, np.float64)
    if N == 0:
        return out
    wk = np.zeros(4 * (N + 1), np.float64)
    lib().orc_ray_messages(N, _p(L), _p(ln), float(log_nu_bg), _p(out), _p(wk))
    return out


def ray_messages_divfree(L, log_nu_v, log_nu_bg: float) -> np.ndarray:
    L = np.ascontiguousarray(L, np.float64)
    ln = np.ascontiguousarray(log_nu_v, np.float64)
    out = np.zeros(len(L), np.float64)
    if len(L):
        lib().orc_ray_messages_divfree(len(L), _p(L), _p(ln), float(log_nu_bg), _p(out))
    return out


def transpose(vox, V: int):
    vox = np.ascontiguousarray(vox, np.uint32)
    vstart = np.zeros(V + 1, np.int64)
    eid = np.zeros(max(len(vox), 1), np.int64)
    lib().orc_transpose(len(vox), _p(vox), int(V), _p(vstart), _p(eid))
    return vstart, eid[:len(vox)]


def bp(ray_off, vox, log_nu_e, V: int, prior: float, init_p: float, log_nu_bg: float, iters: int):
    """Flooding loopy BP; returns (lam[E], T[V], p[V]) in FP64."""
    ray_off = np.ascontiguousarray(ray_off, np.int64)
    vox = np.ascontiguousarray(vox, np.uint32)
    ln = np.ascontiguousarray(log_nu_e, np.float64)
    E = int(ray_off[-1])
    assert len(vox) == E and len(ln) == E
    lam = np.zeros(max(E, 1), np.float64)
    T = np.zeros(V, np.float64)
    p = np.zeros(V, np.float64)
    rc = lib().orc_bp(len(ray_off) - 1, _p(ray_off), _p(vox if E else np.zeros(1, np.uint32)),
                      _p(ln if E else np.zeros(1)), int(V), float(prior), float(init_p),
                      float(log_nu_bg), int(iters), _p(lam), _p(T), _p(p))
    if rc != 0:
        raise MemoryError("oracle bp allocation failed")
    return lam[:E], T, p


def bp_variants(ray_off, vox, log_nu_e, V: int, prior: float, init_p: float, log_nu_bg: float, iters: int,
                wlen=None, ray_frame=None):
    """Flooding BP with the implementation's variants (mrf_oracle.c section 8): traversed-length weights
    wlen[E] and/or per-keyframe average messages (ray_frame[R], non-decreasing).  Returns (stored per-edge
    values, T, p)."""
    ray_off = np.ascontiguousarray(ray_off, np.int64)
    vox = np.ascontiguousarray(vox, np.uint32)
    ln = np.ascontiguousarray(log_nu_e, np.float64)
    E = int(ray_off[-1])
    R = len(ray_off) - 1
    wl = None if wlen is None else np.ascontiguousarray(wlen, np.float64)
    rf = None if ray_frame is None else np.ascontiguousarray(ray_frame, np.int32)
    assert wl is None or len(wl) == E
    assert rf is None or len(rf) == R
    lam = np.zeros(max(E, 1), np.float64)
    T = np.zeros(V, np.float64)
    p = np.zeros(V, np.float64)
    rc = lib().orc_bp_variants(R, _p(ray_off), _p(vox if E else np.zeros(1, np.uint32)),
                               _p(ln if E else np.zeros(1)), int(V), float(prior), float(init_p),
                               float(log_nu_bg), int(iters), None if wl is None else _p(wl),
                               None if rf is None else _p(rf), _p(lam), _p(T), _p(p))
    if rc == -2:
        raise ValueError("ray_frame must be non-decreasing")
    if rc != 0:
        raise MemoryError("oracle bp allocation failed")
    return lam[:E], T, p


def infer_variants(workload, length_weight: bool = False, keyframe_avg: bool = False, iters=None):
    """Oracle marginals of a synth.Workload under the implementation's variants: dict(p, T, lam)."""
    csr = trace_frames(workload.grid, workload.frames, workload.lut)
    ln = log_nu_edges(workload.lut, csr["ray_off"], csr["Z"], csr["d"])
    wl = length_weights(workload.grid, workload.frames, workload.lut) if length_weight else None
    rf = None
    if keyframe_avg:
        rf = np.concatenate([np.full(fr.cam.W * fr.cam.H, k, np.int32) for k, fr in enumerate(workload.frames)])
    ip = workload.init_p or workload.prior
    it = workload.iters if iters is None else iters
    lam, T, p = bp_variants(csr["ray_off"], csr["vox"], ln, workload.grid.n_voxels, workload.prior, ip,
                            default_log_nu_bg(workload.lut), it, wl, rf)
    return dict(p=p, T=T, lam=lam)


# --------------------------------------------------------------------------
# whole workloads
# --------------------------------------------------------------------------
def trace_frames(grid, frames, lut):
    """Concatenate the CSR of several frames (ray ids frame-major, row-major pixels)."""
    offs, voxs, ds, Zs = [np.zeros(1, np.int64)], [], [], []
    base = 0
    for fr in frames:
        t = trace_frame(grid, fr.cam, fr.depth, lut)
        offs.append(t["ray_off"][1:] + base)
        base += int(t["ray_off"][-1])
        voxs.append(t["vox"])
        ds.append(t["d"])
        Zs.append(t["Z"])
    return dict(ray_off=np.concatenate(offs), vox=np.concatenate(voxs) if voxs else np.zeros(0, np.uint32),
                d=np.concatenate(ds) if ds else np.zeros(0, np.float32),
                Z=np.concatenate(Zs) if Zs else np.zeros(0, np.float32))


def infer(workload, iters=None, init_p=None, log_nu_bg=None, frames=None):
    """Oracle marginals for a synth.Workload: dict(p, T, lam, csr, log_nu)."""
    frames = workload.frames if frames is None else frames
    csr = trace_frames(workload.grid, frames, workload.lut)
    ln = log_nu_edges(workload.lut, csr["ray_off"], csr["Z"], csr["d"])
    lbg = default_log_nu_bg(workload.lut) if log_nu_bg is None else log_nu_bg
    it = workload.iters if iters is None else iters
    ip = workload.prior if init_p is None else init_p
    lam, T, p = bp(csr["ray_off"], csr["vox"], ln, workload.grid.n_voxels, workload.prior, ip, lbg, it)
    return dict(p=p, T=T, lam=lam, csr=csr, log_nu=ln)


# --------------------------------------------------------------------------
# differentiation with respect to the noise table (see mrf_oracle.c section 6)
# --------------------------------------------------------------------------
def nu_theta_edges(lut, ls_tab, w: float, ray_off, Z, d) -> np.ndarray:
    """Linear likelihoods nu of every edge with the table's log sigma replaced by ls_tab (FP64) and weight w."""
    ray_off = np.ascontiguousarray(ray_off, np.int64)
    Z = np.ascontiguousarray(Z, np.float32)
    d = np.ascontiguousarray(d, np.float32)
    ls = np.ascontiguousarray(ls_tab, np.float64)
    out = np.zeros(max(len(d), 1), np.float64)
    lh = _LutHold(lut)
    lib().orc_nu_theta_edges(C.byref(lh.s), _p(ls), float(w), len(ray_off) - 1, _p(ray_off), _p(Z), _p(d), _p(out))
    return out[:len(d)]


def heldout_loss(ray_off, vox, nu, nu_bg: float, p, grad: bool = False):
    """-sum_r log S_r (held-out depth likelihood under the marginals p); with grad, also d/dp, d/dnu, d/dnu_bg."""
    ray_off = np.ascontiguousarray(ray_off, np.int64)
    vox = np.ascontiguousarray(vox, np.uint32)
    nu = np.ascontiguousarray(nu, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    if not grad:
        return float(lib().orc_heldout_loss(len(ray_off) - 1, _p(ray_off), _p(vox), _p(nu), float(nu_bg), _p(p),
                                            None, None, None))
    gp = np.zeros(len(p), np.float64)
    gnu = np.zeros(max(len(nu), 1), np.float64)
    gbg = np.zeros(1, np.float64)
    loss = lib().orc_heldout_loss(len(ray_off) - 1, _p(ray_off), _p(vox), _p(nu), float(nu_bg), _p(p), _p(gp),
                                  _p(gnu), _p(gbg))
    return float(loss), gp, gnu[:len(nu)], float(gbg[0])


def ray_messages_adjoint(L, nu, nu_bg: float, g):
    """Reverse mode of ray_messages for one ray: (d/dL, d/dnu (linear), d/dnu_bg) given g = d loss / d lambda."""
    L = np.ascontiguousarray(L, np.float64)
    nu = np.ascontiguousarray(nu, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    N = len(L)
    gL = np.zeros(N, np.float64)
    gnu = np.zeros(N, np.float64)
    gbg = np.zeros(1, np.float64)
    work = np.zeros(9 * (N + 1), np.float64)
    lib().orc_ray_messages_adjoint(N, _p(L), _p(nu), float(nu_bg), _p(g), _p(gL), _p(gnu), _p(gbg), _p(work))
    return gL, gnu, float(gbg[0])


def grad(lut, ls_tab, w: float, train, heldout, V: int, prior: float, init_p: float, iters: int,
         with_grad: bool = True):
    """Held-out loss after `iters` BP passes on the training edges, and (with_grad) its gradient with respect to
    the table theta = (ls_tab, w); nu_bg = w / d_hi.  train / heldout are CSR dicts (ray_off, vox, d, Z) as from
    trace_frames.  Returns loss, or (loss, g_ls[n_bins], g_w)."""
    ls = np.ascontiguousarray(ls_tab, np.float64)
    assert len(ls) == lut.n_bins
    a = [np.ascontiguousarray(train["ray_off"], np.int64), np.ascontiguousarray(train["vox"], np.uint32),
         np.ascontiguousarray(train["d"], np.float32), np.ascontiguousarray(train["Z"], np.float32),
         np.ascontiguousarray(heldout["ray_off"], np.int64), np.ascontiguousarray(heldout["vox"], np.uint32),
         np.ascontiguousarray(heldout["d"], np.float32), np.ascontiguousarray(heldout["Z"], np.float32)]
    a = [x if len(x) else np.zeros(1, x.dtype) for x in a]
    loss = np.zeros(1, np.float64)
    g_ls = np.zeros(lut.n_bins, np.float64)
    g_w = np.zeros(1, np.float64)
    lh = _LutHold(lut)
    rc = lib().orc_grad(C.byref(lh.s), _p(ls), float(w), len(train["ray_off"]) - 1, _p(a[0]), _p(a[1]), _p(a[2]),
                        _p(a[3]), len(heldout["ray_off"]) - 1, _p(a[4]), _p(a[5]), _p(a[6]), _p(a[7]), int(V),
                        float(prior), float(init_p), int(iters), _p(loss), _p(g_ls) if with_grad else None,
                        _p(g_w))
    if rc != 0:
        raise MemoryError("oracle grad allocation failed")
    return (float(loss[0]), g_ls, float(g_w[0])) if with_grad else float(loss[0])


# --------------------------------------------------------------------------
# evaluation metric (mrf_oracle.c section 7)
# --------------------------------------------------------------------------
def omega_ray(vox, t_in, t_out, p, h: float, Z: float):
    """Classification of one ray walked to the map boundary: (accurate 0/1, chosen voxel index or -1)."""
    vox = np.ascontiguousarray(vox, np.uint32)
    ti = np.ascontiguousarray(t_in, np.float32)
    to = np.ascontiguousarray(t_out, np.float32)
    p = np.ascontiguousarray(p, np.float64)
    ch = C.c_int()
    acc = lib().orc_omega_ray(len(vox), _p(vox), _p(ti), _p(to), _p(p), float(h), float(Z), C.byref(ch))
    return int(acc), ch.value


def omega_frame(grid, cam, lut, depth, p):
    """Per pixel of a frame: 1 accurate, 0 not, -1 not evaluated (invalid depth or a ray missing the grid),
    against marginals p of the nx*ny*nz voxels (x fastest)."""
    depth = np.ascontiguousarray(depth, np.float32)
    p = np.ascontiguousarray(np.asarray(p, np.float64).ravel())
    out = np.zeros(cam.W * cam.H, np.int8)
    g, cm, lh = _grid(grid), _cam(cam), _LutHold(lut)
    lib().orc_omega_frame(C.byref(g), C.byref(cm), C.byref(lh.s), _p(depth), _p(p), _p(out))
    return out
