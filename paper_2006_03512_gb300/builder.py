"""Compile the CUDA library (libmrfmap.so) for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library with an rpath to the toolkit's runtime.  traverse.cu is compiled with
-fmad=false (and IEEE division / square root, nvcc's default) so that the
3D-DDA recipe rounds exactly as written.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmrfmap.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = {
    "traverse.cu": ["-fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "scan.cu": [],
    "sort.cu": [],
    "bp.cu": [],
    "ray_pipe.cu": [],
    "group.cu": [],
    "grad.cu": [],
    "noalloc.cu": [],
    "api.cu": [],
}


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _cuda_lib_dir() -> str:
    nvcc = os.path.realpath(_nvcc())
    home = os.path.dirname(os.path.dirname(nvcc))
    for sub in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"), os.path.join("targets", "x86_64-linux", "lib")):
        d = os.path.join(home, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")) or os.path.exists(os.path.join(d, "libcudart.so.13")):
            return d
    return os.path.join(home, "lib64")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in ("mrf_internal.cuh", "ray_tile.cuh", "seg_scan.cuh", "async_copy.cuh")]
    headers += [os.path.join(INC, "mrfmap.h"), __file__]
    objs, jobs = [], []
    for src, flags in SOURCES.items():
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
                   *flags, *extra_flags, "-c", s, "-o", o]
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            if res.returncode != 0:
                raise RuntimeError("nvcc failed for " + cmd[-3])
    if force or jobs or _stale(LIB, objs):
        libdir = _cuda_lib_dir()
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-L", libdir,
               "-Xlinker", "-rpath=" + libdir]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
