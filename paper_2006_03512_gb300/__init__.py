"""GB300 (sm_103a) ray-MRF occupancy mapping: Python binding of libmrfmap.so.

Argument marshalling only.  Every step of the mapping path (ray set-up, 3D-DDA
traversal, transpose, ray->voxel messages, voxel totals, marginals) runs in
the library's CUDA kernels; PyTorch supplies device memory and the stream.
Importing this module does not build anything; ``build()`` compiles the
library, and every entry point raises if it has not been built.

The C ABI is declared in include/mrfmap.h; the names here mirror it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmrfmap.so")

MRF_OK, MRF_EINVAL, MRF_ENOMEM, MRF_ECUDA, MRF_ETIMEOUT, MRF_ESTATE, MRF_ERANGE = 0, -1, -2, -3, -4, -5, -6
PREC_F32, PREC_F64, PREC_BF16, PREC_F32_LOG = 0, 1, 2, 3
VAR_LENGTH_WEIGHT, VAR_KEYFRAME_AVG = 1, 2
_CODES = {0: "MRF_OK", -1: "MRF_EINVAL", -2: "MRF_ENOMEM", -3: "MRF_ECUDA", -4: "MRF_ETIMEOUT",
          -5: "MRF_ESTATE", -6: "MRF_ERANGE"}

_lock = threading.Lock()
_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libmrfmap.so for sm_103a (nvcc)."""
    from . import builder as _b
    return _b.build(force=force, verbose=verbose)


class MRFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("res", C.c_float),
                ("origin", C.c_float * 3)]


class _Intr(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float)]


class _Lut(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("d_lo", C.c_float), ("d_hi", C.c_float), ("log_sigma", C.c_void_p),
                ("outlier_w", C.c_float), ("bias", C.c_void_p)]


class _Opt(C.Structure):
    _fields_ = [("precision", C.c_int32), ("nu_bg", C.c_float), ("init_p", C.c_float), ("debug_checks", C.c_int32),
                ("variants", C.c_int32), ("long_ray_f64", C.c_int32)]


class ProfileTimes(C.Structure):
    _fields_ = [("ms_ray_messages", C.c_double), ("ms_voxel_reduce", C.c_double), ("ms_other_infer", C.c_double),
                ("ms_build", C.c_double), ("ms_traverse", C.c_double), ("n_ray_messages", C.c_int64),
                ("n_voxel_reduce", C.c_int64), ("n_other_infer", C.c_int64), ("n_build", C.c_int64),
                ("n_traverse", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol declared in include/mrfmap.h, with its ctypes signature
P, I32, I64, F32, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_size_t
SIGNATURES = {
    "mrf_default_options": (None, [P]),
    "mrf_create": (C.c_int, [P, P, F32, P, P]),
    "mrf_destroy": (None, [P]),
    "mrf_reset": (C.c_int, [P]),
    "mrf_set_stream": (C.c_int, [P, P]),
    "mrf_add_frame": (C.c_int, [P, P, I32, I32, P, P, P]),
    "mrf_add_frame_host": (C.c_int, [P, P, I32, I32, P, P, P]),
    "mrf_infer": (C.c_int, [P, I32]),
    "mrf_marginals": (C.c_int, [P, P]),
    "mrf_marginals_host": (C.c_int, [P, P]),
    "mrf_stats": (C.c_int, [P, P, P]),
    "mrf_stats2": (C.c_int, [P, P, P]),
    "mrf_plan_info": (C.c_int, [P, P, P, P]),
    "mrf_add_heldout": (C.c_int, [P, P, C.c_int32, C.c_int32, P, P, P]),
    "mrf_grad": (C.c_int, [P, C.c_int32, P, P, P, P]),
    "mrf_accuracy": (C.c_int, [P, P, I32, I32, P, P, P, P, P, P]),
    "mrf_debug_fail_alloc": (C.c_int, [P, I64]),
    "mrf_debug_wait_probe": (C.c_int, [P]),
    "mrf_create_batch": (C.c_int, [P, I32, P, F32, P, P]),
    "mrf_scene_count": (C.c_int, [P, P, P]),
    "mrf_add_frame_to": (C.c_int, [P, I32, P, I32, I32, P, P, P]),
    "mrf_set_plan": (C.c_int, [P, I32, I32, I32]),
    "mrf_infer_graph": (C.c_int, [P, I32]),
    "mrf_synchronize": (C.c_int, [P]),
    "mrf_last_error": (C.c_char_p, [P]),
    "mrf_export_rays": (C.c_int, [P, P, P, P, P]),
    "mrf_export_nu": (C.c_int, [P, P]),
    "mrf_export_messages": (C.c_int, [P, P, P]),
    "mrf_export_messages_f64": (C.c_int, [P, P, P]),
    "mrf_export_transpose": (C.c_int, [P, P, P, P, P]),
    "mrf_export_groups": (C.c_int, [P, P, P, P, P, P, P, P, P]),
    "mrf_profile_enable": (C.c_int, [P, I32]),
    "mrf_profile_read": (C.c_int, [P, P]),
    "mrf_launch_count": (I64, [P]),
    "mrf_ray_messages_workspace": (SZ, [I64, I64, I32]),
    "mrf_ray_messages": (C.c_int, [P, I64, I32, P, P, P, P, F32, I32, F32, P, SZ, P]),
    "mrf_voxel_reduce_workspace": (SZ, [I64]),
    "mrf_voxel_reduce": (C.c_int, [P, P, P, I64, I64, P, F32, P, P, SZ, P]),
    "mrf_voxel_reduce_noalloc": (C.c_int, [P, P, P, I64, I64, P, F32, P, P]),
}
NOALLOC_MAX_EDGES = 1 << 28


def lib():
    """Load libmrfmap.so; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing); call "
                                   "paper_2006_03512_gb300.build() first")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _dptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _check_cuda(t, dtype, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")


@dataclass
class Options:
    precision: int = PREC_F32
    nu_bg: float = -1.0      # < 0: outlier_w / d_hi of the first frame's table
    init_p: float = 0.0      # <= 0: the prior
    debug_checks: bool = False
    variants: int = 0        # VAR_LENGTH_WEIGHT | VAR_KEYFRAME_AVG (the paper implementation's variants)
    long_ray_f64: int = 0    # > 0: rays longer than this many edges get FP64 prefix/suffix accumulations


class _LutHold:
    """Keeps the host arrays of a noise table alive across a call."""

    def __init__(self, lut):
        self.ls = np.ascontiguousarray(lut.log_sigma, np.float32)
        bias = getattr(lut, "bias", None)
        self.bias = None if bias is None else np.ascontiguousarray(bias, np.float32)
        self.s = _Lut(int(lut.n_bins), float(lut.d_lo), float(lut.d_hi), self.ls.ctypes.data,
                      float(lut.outlier_w), 0 if self.bias is None else self.bias.ctypes.data)


def _pose12(pose) -> "C.Array":
    p = np.ascontiguousarray(np.asarray(pose, np.float64).reshape(12))
    return (C.c_double * 12)(*p.tolist())


class Map:
    """One occupancy map on the current CUDA device (mrf_create / mrf_destroy)."""

    def __init__(self, grid, prior: float, options: Optional[Options] = None, stream=None):
        """grid: one grid, or a list of grids for a batched context (mrf_create_batch)."""
        L = lib()
        torch = _torch()
        grids = list(grid) if isinstance(grid, (list, tuple)) else [grid]
        self.grids = grids
        self.grid = grids[0]
        self.n_scenes = len(grids)
        self.scene_shapes = [(int(g.nz), int(g.ny), int(g.nx)) for g in grids]
        self.scene_voxels = [int(g.nx) * int(g.ny) * int(g.nz) for g in grids]
        self.n_voxels = sum(self.scene_voxels)
        self.shape = self.scene_shapes[0] if self.n_scenes == 1 else (self.n_voxels,)
        self.prior = float(prior)
        opt = options or Options()
        self.options = opt
        self._stream = stream
        self.device = torch.cuda.current_device()
        gs = (_Grid * len(grids))(*[_Grid(int(g.nx), int(g.ny), int(g.nz), float(g.res),
                                          (C.c_float * 3)(*[float(x) for x in g.origin])) for g in grids])
        o = _Opt(int(opt.precision), float(opt.nu_bg), float(opt.init_p), int(bool(opt.debug_checks)),
                 int(opt.variants), int(opt.long_ray_f64))
        h = C.c_void_p()
        if self.n_scenes == 1:
            rc = L.mrf_create(C.byref(h), gs, float(prior), C.byref(o), _stream_handle(stream))
        else:
            rc = L.mrf_create_batch(C.byref(h), len(grids), gs, float(prior), C.byref(o), _stream_handle(stream))
        if rc != MRF_OK:
            raise MRFError(rc, "mrf_create failed")
        self._h = h

    def scene_marginals(self, p, scene: int):
        """View of scene `scene` (nz, ny, nx) inside the marginals of a batched context."""
        a = sum(self.scene_voxels[:scene])
        return p.reshape(-1)[a:a + self.scene_voxels[scene]].reshape(self.scene_shapes[scene])

    def set_plan(self, ray_items: int = 0, threads: int = 0, groups: int = -1):
        """Kernel plan for the next build (mrf_set_plan): 0 / -1 leave the choice to the library."""
        self._rc(lib().mrf_set_plan(self._h, int(ray_items), int(threads), int(groups)), "mrf_set_plan")

    def infer_graph(self, iters: int):
        """mrf_infer recorded once as a CUDA graph and replayed (mrf_infer_graph)."""
        self._rc(lib().mrf_infer_graph(self._h, int(iters)), "mrf_infer_graph")

    # -- plumbing
    def _rc(self, rc: int, what: str):
        if rc != MRF_OK:
            msg = lib().mrf_last_error(self._h).decode()
            raise MRFError(rc, f"{what}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            lib().mrf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        self._stream = stream
        self._rc(lib().mrf_set_stream(self._h, _stream_handle(stream)), "mrf_set_stream")

    # -- API
    def reset(self):
        self._rc(lib().mrf_reset(self._h), "mrf_reset")

    def add_frame(self, depth, pose, intrinsics, lut, scene: int = 0):
        """depth: (H, W) float32 z-depths, a CUDA tensor (device) or a numpy array (host, scene 0)."""
        K = _Intr(float(intrinsics.fx), float(intrinsics.fy), float(intrinsics.cx), float(intrinsics.cy))
        lh = _LutHold(lut)
        pz = _pose12(pose)
        if scene:
            _check_cuda(depth, _torch().float32, "depth")
            H, W = depth.shape
            rc = lib().mrf_add_frame_to(self._h, int(scene), _dptr(depth), W, H, pz, C.byref(K), C.byref(lh.s))
            self._rc(rc, "mrf_add_frame_to")
            return
        if isinstance(depth, np.ndarray):
            d = np.ascontiguousarray(depth, np.float32)
            H, W = d.shape
            rc = lib().mrf_add_frame_host(self._h, d.ctypes.data, W, H, pz, C.byref(K), C.byref(lh.s))
            self._rc(rc, "mrf_add_frame_host")
        else:
            _check_cuda(depth, _torch().float32, "depth")
            H, W = depth.shape
            rc = lib().mrf_add_frame(self._h, _dptr(depth), W, H, pz, C.byref(K), C.byref(lh.s))
            self._rc(rc, "mrf_add_frame")

    def infer(self, iters: int):
        self._rc(lib().mrf_infer(self._h, int(iters)), "mrf_infer")

    def add_heldout(self, depth, pose, intrinsics, lut):
        """A held-out depth frame (CUDA tensor (H, W) float32) for grad(); kept out of the map."""
        K = _Intr(float(intrinsics.fx), float(intrinsics.fy), float(intrinsics.cx), float(intrinsics.cy))
        lh = _LutHold(lut)
        _check_cuda(depth, _torch().float32, "depth")
        H, W = depth.shape
        rc = lib().mrf_add_heldout(self._h, _dptr(depth), W, H, _pose12(pose), C.byref(K), C.byref(lh.s))
        self._rc(rc, "mrf_add_heldout")

    def accuracy(self, depth, pose, intrinsics, lut, per_pixel: bool = False):
        """The paper's accuracy metric of the current marginals on one depth frame (CUDA tensor (H, W)
        float32), rays walked to the grid exit (mrf_accuracy): returns (accurate rays, evaluated rays), and
        with per_pixel also the int8 (H, W) tensor of 1 accurate / 0 not / -1 not evaluated."""
        torch = _torch()
        K = _Intr(float(intrinsics.fx), float(intrinsics.fy), float(intrinsics.cx), float(intrinsics.cy))
        lh = _LutHold(lut)
        _check_cuda(depth, torch.float32, "depth")
        H, W = depth.shape
        res = torch.empty((H, W), dtype=torch.int8, device=depth.device) if per_pixel else None
        n_acc, n_ev = C.c_int64(), C.c_int64()
        rc = lib().mrf_accuracy(self._h, _dptr(depth), W, H, _pose12(pose), C.byref(K), C.byref(lh.s),
                                _dptr(res) if per_pixel else None, C.byref(n_acc), C.byref(n_ev))
        self._rc(rc, "mrf_accuracy")
        return (n_acc.value, n_ev.value, res) if per_pixel else (n_acc.value, n_ev.value)

    def debug_fail_alloc(self, nth: int):
        """Failure injection: the nth device allocation from now fails with MRF_ENOMEM (0: off)."""
        self._rc(lib().mrf_debug_fail_alloc(self._h, int(nth)), "mrf_debug_fail_alloc")

    def debug_wait_probe(self):
        """Enqueue a bounded device-side wait that times out (the next synchronize raises MRF_ETIMEOUT)."""
        self._rc(lib().mrf_debug_wait_probe(self._h), "mrf_debug_wait_probe")

    def grad(self, iters: int, theta):
        """Held-out loss and its gradient with respect to the noise table theta (mrf_grad):
        returns (loss, d loss / d log_sigma [n_bins] float64, d loss / d outlier_w)."""
        lh = _LutHold(theta)
        loss = C.c_double()
        g_ls = np.zeros(int(theta.n_bins), np.float64)
        g_w = C.c_double()
        rc = lib().mrf_grad(self._h, int(iters), C.byref(lh.s), C.byref(loss), g_ls.ctypes.data, C.byref(g_w))
        self._rc(rc, "mrf_grad")
        return loss.value, g_ls, g_w.value

    def marginals(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=f"cuda:{self.device}")
        _check_cuda(out, torch.float32, "out")
        self._rc(lib().mrf_marginals(self._h, _dptr(out)), "mrf_marginals")
        return out

    def marginals_host(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == self.n_voxels
        self._rc(lib().mrf_marginals_host(self._h, out.ctypes.data), "mrf_marginals_host")
        return out

    def stats(self):
        r, e = C.c_int64(), C.c_int64()
        self._rc(lib().mrf_stats(self._h, C.byref(r), C.byref(e)), "mrf_stats")
        ml, nt = C.c_int32(), C.c_int64()
        self._rc(lib().mrf_stats2(self._h, C.byref(ml), C.byref(nt)), "mrf_stats2")
        return {"n_rays": r.value, "n_edges": e.value, "max_ray_len": ml.value, "n_touched": nt.value}

    def plan_info(self):
        """Edges per ray-kernel thread, ray tiles and (tile, voxel) groups (0: no grouping)."""
        kt, nt, ng = C.c_int32(), C.c_int64(), C.c_int64()
        self._rc(lib().mrf_plan_info(self._h, C.byref(kt), C.byref(nt), C.byref(ng)), "mrf_plan_info")
        return {"ray_items": kt.value, "n_ray_tiles": nt.value, "n_groups": ng.value}

    def synchronize(self):
        self._rc(lib().mrf_synchronize(self._h), "mrf_synchronize")

    def export_rays(self):
        torch = _torch()
        st = self.stats()
        dev = f"cuda:{self.device}"
        ro = torch.empty(st["n_rays"] + 1, dtype=torch.int64, device=dev)
        vox = torch.empty(max(st["n_edges"], 1), dtype=torch.int32, device=dev)
        d = torch.empty(max(st["n_edges"], 1), dtype=torch.float32, device=dev)
        Z = torch.empty(max(st["n_rays"], 1), dtype=torch.float32, device=dev)
        self._rc(lib().mrf_export_rays(self._h, _dptr(ro), _dptr(vox), _dptr(d), _dptr(Z)), "mrf_export_rays")
        E, R = st["n_edges"], st["n_rays"]
        return {"ray_off": ro, "vox": vox[:E], "d": d[:E], "Z": Z[:R]}

    def export_nu(self):
        torch = _torch()
        E = self.stats()["n_edges"]
        nu = torch.empty(max(E, 1), dtype=torch.float32, device=f"cuda:{self.device}")
        self._rc(lib().mrf_export_nu(self._h, _dptr(nu)), "mrf_export_nu")
        return nu[:E]

    def export_messages(self):
        torch = _torch()
        E = self.stats()["n_edges"]
        dev = f"cuda:{self.device}"
        if self.options.precision == PREC_F64:
            lam = torch.empty(max(E, 1), dtype=torch.float64, device=dev)
            T = torch.empty(self.n_voxels, dtype=torch.float64, device=dev)
            self._rc(lib().mrf_export_messages_f64(self._h, _dptr(lam), _dptr(T)), "mrf_export_messages_f64")
        else:
            lam = torch.empty(max(E, 1), dtype=torch.float32, device=dev)
            T = torch.empty(self.n_voxels, dtype=torch.float32, device=dev)
            self._rc(lib().mrf_export_messages(self._h, _dptr(lam), _dptr(T)), "mrf_export_messages")
        return lam[:E], T

    def export_transpose(self):
        torch = _torch()
        n = C.c_int64()
        self._rc(lib().mrf_export_transpose(self._h, None, None, None, C.byref(n)), "mrf_export_transpose")
        E = self.stats()["n_edges"]
        dev = f"cuda:{self.device}"
        perm = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
        so = torch.empty(n.value + 1, dtype=torch.int32, device=dev)
        sv = torch.empty(max(n.value, 1), dtype=torch.int32, device=dev)
        self._rc(lib().mrf_export_transpose(self._h, _dptr(perm), _dptr(so), _dptr(sv), C.byref(n)),
                 "mrf_export_transpose")
        return {"perm": perm[:E], "seg_off": so, "seg_vox": sv[:n.value]}

    def export_groups(self):
        """The per-tile voxel groups (mrf_export_groups): tile_E, tg_off, lidx, gid, ends, gkey."""
        torch = _torch()
        nt, ng = C.c_int64(), C.c_int64()
        self._rc(lib().mrf_export_groups(self._h, None, None, None, None, None, None, C.byref(nt), C.byref(ng)),
                 "mrf_export_groups")
        E = self.stats()["n_edges"]
        dev = f"cuda:{self.device}"
        out = {"tile_E": torch.empty(nt.value + 1, dtype=torch.int64, device=dev),
               "tg_off": torch.empty(nt.value + 1, dtype=torch.int64, device=dev),
               "lidx": torch.empty(max(E, 1), dtype=torch.int16, device=dev),
               "gid": torch.empty(max(E, 1), dtype=torch.int16, device=dev),
               "ends": torch.empty(max((E + 31) // 32, 1), dtype=torch.int32, device=dev),
               "gkey": torch.empty(max(ng.value, 1), dtype=torch.int32, device=dev)}
        self._rc(lib().mrf_export_groups(self._h, *[_dptr(out[k]) for k in ("tile_E", "tg_off", "lidx", "gid", "ends",
                                                                             "gkey")], C.byref(nt), C.byref(ng)),
                 "mrf_export_groups")
        out["lidx"], out["gid"] = out["lidx"][:E], out["gid"][:E]
        out["ends"], out["gkey"] = out["ends"][:(E + 31) // 32], out["gkey"][:ng.value]
        return out

    def profile(self, on: bool = True):
        self._rc(lib().mrf_profile_enable(self._h, int(bool(on))), "mrf_profile_enable")

    def profile_read(self) -> dict:
        t = ProfileTimes()
        self._rc(lib().mrf_profile_read(self._h, C.byref(t)), "mrf_profile_read")
        return t.as_dict()

    def launch_count(self) -> int:
        return int(lib().mrf_launch_count(self._h))


# --------------------------------------------------------------------------
# standalone kernels on caller tensors
# --------------------------------------------------------------------------
def ray_messages(ray_off, vox, nu, T, lam, nu_bg: float, first: bool = False, L0: float = 0.0,
                 max_ray_len: Optional[int] = None, stream=None):
    """In-place ray->voxel messages (mrf_ray_messages) on CUDA tensors."""
    torch = _torch()
    _check_cuda(ray_off, torch.int64, "ray_off")
    R = ray_off.numel() - 1
    if max_ray_len is None:
        max_ray_len = int((ray_off[1:] - ray_off[:-1]).max().item()) if R > 0 else 0
    E = int(ray_off[-1].item()) if R >= 0 else 0
    ws_b = int(lib().mrf_ray_messages_workspace(R, E, int(max_ray_len)))
    ws = torch.empty(max(ws_b, 16), dtype=torch.uint8, device=ray_off.device)
    rc = lib().mrf_ray_messages(_dptr(ray_off), R, int(max_ray_len), _dptr(vox), _dptr(nu), _dptr(T), _dptr(lam),
                                float(nu_bg), int(bool(first)), float(L0), _dptr(ws), ws_b, _stream_handle(stream))
    if rc != MRF_OK:
        raise MRFError(rc, "mrf_ray_messages")
    return lam


def voxel_reduce(perm, seg_off, seg_vox, lam, logit_prior: float, T, stream=None):
    """T[seg_vox[s]] = logit_prior + sum of lam over segment s (mrf_voxel_reduce)."""
    torch = _torch()
    E = perm.numel()
    S = seg_vox.numel()
    ws_b = int(lib().mrf_voxel_reduce_workspace(E))
    ws = torch.empty(max(ws_b, 16), dtype=torch.uint8, device=perm.device)
    rc = lib().mrf_voxel_reduce(_dptr(perm), _dptr(seg_off), _dptr(seg_vox), S, E, _dptr(lam), float(logit_prior),
                                _dptr(T), _dptr(ws), ws_b, _stream_handle(stream))
    if rc != MRF_OK:
        raise MRFError(rc, "mrf_voxel_reduce")
    return T


def voxel_reduce_noalloc(perm, seg_off, seg_vox, lam, logit_prior: float, T, stream=None):
    """As voxel_reduce, with the library's static scratch (mrf_voxel_reduce_noalloc): no allocation."""
    rc = lib().mrf_voxel_reduce_noalloc(_dptr(perm), _dptr(seg_off), _dptr(seg_vox), seg_vox.numel(), perm.numel(),
                                        _dptr(lam), float(logit_prior), _dptr(T), _stream_handle(stream))
    if rc != MRF_OK:
        raise MRFError(rc, "mrf_voxel_reduce_noalloc")
    return T


def logit(p: float) -> float:
    return math.log(p) - math.log1p(-p)


class HeldoutLoss:
    """The held-out loss of a map as a differentiable function of the noise table, for torch:

        loss = HeldoutLoss.apply(log_sigma, outlier_w, mp, iters, table)

    log_sigma: (n_bins,) tensor, outlier_w: 0-d tensor (any device; float32 or float64); table: a noise
    table whose d_lo, d_hi and bias are used.  The forward calls mrf_grad once; the backward scales the
    gradient it returned."""

    @staticmethod
    def _fn():
        torch = _torch()

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, log_sigma, outlier_w, mp, iters, table):
                import dataclasses
                ls = log_sigma.detach().to("cpu", torch.float32).numpy()
                w = float(outlier_w.detach().cpu())
                theta = dataclasses.replace(table, log_sigma=ls, outlier_w=w, n_bins=len(ls))
                loss, g_ls, g_w = mp.grad(iters, theta)
                ctx.save_for_backward(torch.from_numpy(g_ls).to(log_sigma.device, log_sigma.dtype),
                                      torch.tensor(g_w, dtype=outlier_w.dtype, device=outlier_w.device))
                return torch.tensor(loss, dtype=torch.float64, device=log_sigma.device)

            @staticmethod
            def backward(ctx, gout):
                g_ls, g_w = ctx.saved_tensors
                return gout.to(g_ls.dtype) * g_ls, gout.to(g_w.dtype) * g_w, None, None, None

        return _F

    @classmethod
    def apply(cls, log_sigma, outlier_w, mp, iters, table):
        return cls._fn().apply(log_sigma, outlier_w, mp, iters, table)
