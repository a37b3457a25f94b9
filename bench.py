"""Benchmark: ray-voxel BP edge updates per second on one GB300 (or N replicas).

Workload: 30 seeded synthetic 640x480 depth frames (f = 525) on a 1.5 m camera
ring inside a 5.12 m room with 20 boxes and spheres, 256^3 voxels at 0.02 m,
64-bin noise table with a 0.02 outlier floor, 20 BP passes, FP32 messages.

value      edges x passes / (device time of mrf_infer), inputs resident in HBM;
           mrf_infer = initial messages + 20 x (ray->voxel kernel, voxel totals)
e2e        the same metric through the C ABI with HOST buffers: every step
           resets the map, uploads the 30 frames from pinned host memory
           (mrf_add_frame_host: copy, ray set-up, 3D-DDA), builds the
           transpose, runs the 20 passes and reads all marginals back
           (mrf_marginals_host)
roofline   the dominant kernel's algorithmic bytes / its CUDA-event time
cpu_baseline  the FP64 oracle on the host cores, on a bounded sample
           (the first frame of the same workload, same grid and passes)

Multi-GPU (torchrun): replicas only.  Each rank maps the same workload on its
own GPU; no collective touches the data path; value sums the ranks' edge
updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-voxel BP edge updates/sec + % HBM roofline (FP32/batched vs plain FP64 GPU, ≤1e-4 err)"
UNIT = "edge-updates/s"
WORKLOAD = "room_30x640x480"
# algorithmic bytes per edge and pass (FP32): ray kernel reads vox, nu, lambda_old,
# T[vox] and writes lambda_new (20 B); voxel totals read perm and gather lambda (8 B)
BYTES_RAY_EDGE = 20
BYTES_RAY_EDGE_FIRST = 8      # first pass: cavities are the initial message, no vox/lambda/T reads
BYTES_RED_EDGE = 8
BYTES_RED_SEG = 12            # seg_off, seg_vox, T write per non-empty voxel
# with (tile, voxel) groups: the ray kernel also reads each edge's window index
# (u16) and the ray-start and group-end bitmaps, and writes one partial sum per
# group; the voxel totals then read a slot index and gather a partial per group
BYTES_GROUP_EDGE = 2.25
BYTES_GROUP_RAY = 4
BYTES_RED_GROUP = 8
BYTES_F64_EDGE = 48


def _err_summary(torch, p, ref):
    """|p - ref| over all voxels: max, 99.9th and 99.99th percentiles, mean, voxels above 1e-4."""
    d = (p.double() - ref.double()).abs().view(-1)
    srt = torch.sort(d.float()).values
    q = lambda f: float(srt[int(f * (srt.numel() - 1))])
    return {"max": float(d.max()), "p99.9": q(0.999), "p99.99": q(0.9999), "mean": float(d.mean()),
            "n_above_1e-4": int((d > 1e-4).sum())}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2006_03512_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"ray_messages_f32": ["ray_pipe.cu", "ray_tile.cuh"],
                  "voxel_reduce_f32": ["bp.cu", "seg_scan.cuh"]}


def _ncu_traffic(kernel_key):
    """Per-edge DRAM traffic of a kernel from a committed ncu summary, if the source still matches."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[kernel_key]
        if ent.get("source_hash") != _kernel_hash(KERNEL_SOURCES[kernel_key]):
            return None
        return ent
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _reduce_device(dist):
    """Where a scalar all-reduce runs: the GPU under NCCL, the host under gloo."""
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def _barrier_max(torch, dist, world, x: float) -> float:
    """The slowest rank's value (every rank gets it)."""
    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum(torch, dist, world, x: float) -> float:
    """The sum over ranks (every rank gets it)."""
    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(w, n_frames=1):
    """The oracle's own inputs for the bounded CPU sample: the first frame(s)."""
    import oracle
    frames = w.frames[:n_frames]
    csr = oracle.trace_frames(w.grid, frames, w.lut)
    ln = oracle.log_nu_edges(w.lut, csr["ray_off"], csr["Z"], csr["d"])
    return csr, ln


def run_oracle_timed(w, csr, ln, iters):
    import oracle
    t0 = time.perf_counter()
    oracle.bp(csr["ray_off"], csr["vox"], ln, w.grid.n_voxels, w.prior, w.init_p or w.prior,
              oracle.default_log_nu_bg(w.lut), iters)
    return time.perf_counter() - t0


def reference_arm(args):
    """The FP64 CPU oracle timed on the host cores (rank 0 only)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from synth import make_workload
    w = make_workload(WORKLOAD)
    oracle.set_threads(os.cpu_count() or 1)
    csr, ln = oracle_sample(w, 1)
    E = int(csr["ray_off"][-1])
    for _ in range(args.warmup):
        run_oracle_timed(w, csr, ln, args.iters or w.iters)
    ts = [run_oracle_timed(w, csr, ln, args.iters or w.iters) for _ in range(args.steps)]
    it = args.iters or w.iters
    v = E * it * args.steps / sum(ts)
    sample = f"frame 0 of {WORKLOAD} ({E} edges), {it} passes, full 256^3 grid"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _batch_scene(index):
    """One scene of the 64-scene batch, generated in a worker process."""
    from synth.scenes import make_batch_scene
    w = make_batch_scene(index)
    return index, w


def batch_bench(args):
    """The 64-scene batch (uneven grids 64^3-192^3 at 0.03 m, 8-60 frames of 320x240, 15 passes): scenes
    rendered on the host cores, then run in waves of batched contexts (the collection exceeds one
    context's 2^32-edge index and the device memory), each wave's passes replayed as one CUDA graph."""
    import concurrent.futures as cf
    import multiprocessing as mpr
    from synth.scenes import BATCH64_SCENES
    rank, world, local = _dist()
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    # the pool starts (spawn) before this process touches the GPU
    with cf.ProcessPoolExecutor(max_workers=os.cpu_count() or 4, mp_context=mpr.get_context("spawn")) as ex:
        scenes = dict(ex.map(_batch_scene, range(BATCH64_SCENES)))
    gen_s = time.perf_counter() - t0
    import torch
    import paper_2006_03512_gb300 as m
    from paper_2006_03512_gb300 import autotune
    m.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    iters = args.iters or scenes[0].iters
    # waves: about 2.5e9 edges each by the estimate frames * pixels * grid edge
    est = {i: len(w.frames) * 320 * 240 * w.grid.nx for i, w in scenes.items()}
    waves, cur, tot = [], [], 0
    for i in range(BATCH64_SCENES):
        if cur and tot + est[i] > 2.5e9:
            waves.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += est[i]
    waves.append(cur)
    E_all, ms_all, build_ms, plans = 0, 0.0, 0.0, []
    with ClockSampler(local) as clk:
        for wi, idx in enumerate(waves):
            ws = [scenes[i] for i in idx]
            mp = m.Map([w.grid for w in ws], 0.5, m.Options(init_p=ws[0].init_p), stream=stream)
            for s, w in enumerate(ws):
                for fr in w.frames:
                    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut, scene=s)
            plan = None if args.tune else autotune.apply(mp)
            if plan is None:
                plan = tuple(autotune.tune(mp, iters=3)["plan"])
            plans.append(list(plan))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mp.infer(1)                 # builds the transpose
            e1.record(stream)
            torch.cuda.synchronize()
            build_ms += e0.elapsed_time(e1)
            mp.infer_graph(iters)       # records
            for _ in range(max(1, args.warmup - 1)):
                mp.infer_graph(iters)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                mp.infer_graph(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_all += e0.elapsed_time(e1) / args.steps
            E_all += mp.stats()["n_edges"]
            mp.close()
    value = E_all * iters / (ms_all / 1e3)
    peak, peak_kind = _peaks()
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch64", "scenes": BATCH64_SCENES, "waves": len(waves), "passes": iters,
                      "edges": E_all, "plans": plans, "graph": True,
                      "l2": "inputs larger than L2 (per-edge arrays of every wave > 10 GB)"},
           "whole_step_model_frac": (28.0 * E_all * iters / (ms_all / 1e3) / 1e9) / peak, "peak_kind": peak_kind,
           "build_ms": build_ms, "generate_s": gen_s, "clocks": clk.summary()}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--iters", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--no-grad", action="store_true", help="skip the mrf_grad timing")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--frames", type=int, default=0,
                    help="use only the first N frames (small cases for ncu captures; not a bench value)")
    ap.add_argument("--tune", action="store_true", help="batch64: time every kernel plan even if one is stored")
    ap.add_argument("--plan", default="", help="kernel plan 'items,threads,groups' (Map.set_plan) for the timed maps")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the paper implementation's BP variants")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch64":
        return batch_bench(args)

    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2006_03512_gb300 as m
    from synth import make_workload
    m.build()
    w = make_workload(args.workload)
    if args.frames:
        w.frames = w.frames[:args.frames]
    iters = args.iters or w.iters
    stream = torch.cuda.current_stream()

    def sync():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    # ---------------------------------------------------------------- device-resident run
    depths = [torch.from_numpy(fr.depth).cuda() for fr in w.frames]
    opts = dict(init_p=w.init_p)
    plan = tuple(int(x) for x in args.plan.split(",")) if args.plan else None
    mp = m.Map(w.grid, w.prior, m.Options(**opts), stream=stream)
    if plan:
        mp.set_plan(*plan)
    mp.profile(True)
    for d, fr in zip(depths, w.frames):
        mp.add_frame(d, fr.cam.pose, fr.cam, w.lut)
    mp.infer(iters)            # first call builds the transpose
    mp.synchronize()
    prof0 = mp.profile_read()
    st = mp.stats()
    E, S = st["n_edges"], st["n_touched"]
    for _ in range(max(args.warmup - 1, 0)):
        mp.infer(iters)
    if args.steps == 0:   # set-up only (profiling runs that capture the first passes)
        return 0
    mp.profile_read()
    sync()
    launches0 = mp.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        sync()
        ev0.record(stream)
        for _ in range(args.steps):
            mp.infer(iters)
        ev1.record(stream)
        sync()
    launches = mp.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    prof = mp.profile_read()
    ms_max = _barrier_max(torch, dist, world, ms)
    edge_updates = _sum(torch, dist, world, float(E) * iters * args.steps)
    value = edge_updates / (ms_max / 1e3)

    # roofline of the dominant kernel (times from the same timed region)
    peak, peak_kind = _peaks()
    n_ray, n_red = prof["n_ray_messages"], prof["n_voxel_reduce"]
    G = mp.plan_info()["n_groups"]
    ray_bytes = E * (BYTES_RAY_EDGE_FIRST + BYTES_RAY_EDGE * (iters - 1)) * args.steps
    if G > 0:
        ray_bytes += (E * BYTES_GROUP_EDGE + G * BYTES_GROUP_RAY) * iters * args.steps
        red_bytes = (G * BYTES_RED_GROUP + S * BYTES_RED_SEG) * iters * args.steps
    else:
        red_bytes = (E * BYTES_RED_EDGE + S * BYTES_RED_SEG) * iters * args.steps
    ray_gbs = ray_bytes / (prof["ms_ray_messages"] / 1e3) / 1e9
    red_gbs = red_bytes / (prof["ms_voxel_reduce"] / 1e3) / 1e9
    if prof["ms_ray_messages"] >= prof["ms_voxel_reduce"]:
        dom, ach, nl, key = "ray_messages", ray_gbs, n_ray, "ray_messages_f32"
    else:
        dom, ach, nl, key = "voxel_reduce", red_gbs, n_red, "voxel_reduce_f32"
    tr = _ncu_traffic(key)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": peak_kind,
                "traffic": (tr["bytes_per_edge"] * E) if tr else None,
                "algorithmic_bytes_per_launch": (ray_bytes if dom == "ray_messages" else red_bytes) / max(nl, 1),
                "launches": nl,
                "other_kernel": {"ray_messages": {"GB/s": ray_gbs, "ms": prof["ms_ray_messages"]},
                                 "voxel_reduce": {"GB/s": red_gbs, "ms": prof["ms_voxel_reduce"]},
                                 "other_ms": prof["ms_other_infer"]}}
    model_frac = (28.0 * E * iters * args.steps / (ms / 1e3) / 1e9) / peak

    # traversal and transpose throughput (from the first build above)
    extra = {"edges": E, "rays": st["n_rays"], "touched_voxels": S, "max_ray_len": st["max_ray_len"],
             "groups": G,
             "traverse_edges_per_s": E / (prof0["ms_traverse"] / 1e3) if prof0["ms_traverse"] else None,
             "transpose_ms": prof0["ms_build"], "whole_step_model_frac": model_frac}
    p32 = mp.marginals().clone()   # for the error against the FP64 form
    extra["plan"] = mp.plan_info()
    # the paper's accuracy metric of the map on its first frame
    fr0 = w.frames[0]
    acc = {"frame": 0, "fp32": mp.accuracy(depths[0], fr0.cam.pose, fr0.cam, w.lut)}
    mp.close()
    del depths

    # ---------------------------------------------------------------- end to end through the C ABI
    e2e = None
    if not args.no_e2e:
        pinned = []
        for fr in w.frames:
            t = torch.from_numpy(fr.depth).pin_memory()
            pinned.append(t.numpy())
        out = torch.empty(w.grid.n_voxels, dtype=torch.float32).pin_memory().numpy()
        mp = m.Map(w.grid, w.prior, m.Options(**opts), stream=stream)
        if plan:
            mp.set_plan(*plan)

        def step():
            mp.reset()
            for d, fr in zip(pinned, w.frames):
                mp.add_frame(d, fr.cam.pose, fr.cam, w.lut)
            mp.infer(iters)
            mp.marginals_host(out.reshape(mp.shape))

        step()
        sync()
        k = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(k):
            step()
        sync()
        dt = _barrier_max(torch, dist, world, (time.perf_counter() - t0) / k)
        e2e = {"value": _sum(torch, dist, world, float(E) * iters) / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(fr.depth.nbytes for fr in w.frames)),
               "d2h_bytes_per_step": int(w.grid.n_voxels * 4), "ms_per_step": dt * 1e3, "steps": k}
        mp.close()

    # ---------------------------------------------------------------- plain FP64 GPU comparator
    f64 = None
    if not args.no_f64:
        mp = m.Map(w.grid, w.prior, m.Options(precision=m.PREC_F64, **opts), stream=stream)
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
        mp.infer(iters)
        sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mp.infer(iters)
        e1.record(stream)
        sync()
        fms = e0.elapsed_time(e1)
        f64 = {"value": float(E) * iters / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
               "model_GB/s": BYTES_F64_EDGE * E * iters / (fms / 1e3) / 1e9}
        p64 = mp.marginals().clone()
        acc["fp64"] = mp.accuracy(torch.from_numpy(fr0.depth).cuda(), fr0.cam.pose, fr0.cam, w.lut)
        mp.close()
        # the FP64 form's own sensitivity: every log-sigma entry of the noise
        # table moved up by one float32 ulp, a rounding-size change of the
        # likelihoods; voxels where this moves p are where BP amplifies rounding
        lut_b = dataclasses.replace(w.lut, log_sigma=np.nextafter(np.asarray(w.lut.log_sigma, np.float32),
                                                                  np.float32(np.inf)))
        mp = m.Map(w.grid, w.prior, m.Options(precision=m.PREC_F64, **opts), stream=stream)
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, lut_b)
        mp.infer(iters)
        f64["self_sensitivity"] = {"perturbation": "log-sigma table + 1 float32 ulp",
                                   **_err_summary(torch, mp.marginals(), p64)}
        mp.close()
        # bf16 message storage (FP32 arithmetic), timed the same way
        mp = m.Map(w.grid, w.prior, m.Options(precision=m.PREC_BF16, **opts), stream=stream)
        if plan:
            mp.set_plan(*plan)
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
        mp.infer(iters)
        sync()
        e0.record(stream)
        mp.infer(iters)
        e1.record(stream)
        sync()
        bms = e0.elapsed_time(e1)
        p16 = mp.marginals().clone()
        acc["bf16"] = mp.accuracy(torch.from_numpy(fr0.depth).cuda(), fr0.cam.pose, fr0.cam, w.lut)
        mp.close()
        f64["errors_vs_fp64"] = {"fp32": _err_summary(torch, p32, p64), "bf16": _err_summary(torch, p16, p64)}
        # FP64 accumulations on the rays longer than 512 voxels (where there are any), timed the same way
        if st["max_ray_len"] > 512:
            mp = m.Map(w.grid, w.prior, m.Options(long_ray_f64=512, **opts), stream=stream)
            for fr in w.frames:
                mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
            mp.infer(iters)
            sync()
            e0.record(stream)
            mp.infer(iters)
            e1.record(stream)
            sync()
            lms = e0.elapsed_time(e1)
            f64["errors_vs_fp64"]["fp32_long_rays_fp64"] = _err_summary(torch, mp.marginals(), p64)
            f64["long_rays_fp64"] = {"threshold": 512, "value": float(E) * iters / (lms / 1e3), "unit": UNIT,
                                     "ms_per_step": lms}
            mp.close()
        f64["bf16_storage"] = {"value": float(E) * iters / (bms / 1e3), "unit": UNIT, "ms_per_step": bms}
        del p16, p32, p64

    # ---------------------------------------------------------------- the implementation's BP variants
    variants = None
    if not args.no_variants:
        variants = {}
        for name, flag in [("length_weight", m.VAR_LENGTH_WEIGHT), ("keyframe_avg", m.VAR_KEYFRAME_AVG)]:
            mp = m.Map(w.grid, w.prior, m.Options(variants=flag, **opts), stream=stream)
            for fr in w.frames:
                mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
            mp.infer(iters)
            sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mp.infer(iters)
            e1.record(stream)
            sync()
            vms = e0.elapsed_time(e1)
            variants[name] = {"value": float(E) * iters / (vms / 1e3), "unit": UNIT, "ms_per_step": vms,
                              "plan": mp.plan_info()}
            mp.close()

    # ---------------------------------------------------------------- gradient (mrf_grad) on its workload
    grad = None
    if not args.no_grad:
        from synth.scenes import theta_off
        wd = make_workload("diff_8x160x120")
        th = theta_off(wd.lut)
        mp = m.Map(wd.grid, wd.prior, m.Options(init_p=wd.init_p), stream=stream)
        for fr in wd.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, th)
        for fr in wd.heldout:
            mp.add_heldout(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, th)
        mp.grad(wd.iters, th)   # warm-up (builds the transposes)
        ts = []
        for _ in range(3):
            sync()
            t0 = time.perf_counter()
            loss, _, _ = mp.grad(wd.iters, th)
            ts.append(time.perf_counter() - t0)
        Ed = mp.stats()["n_edges"]
        gms = 1e3 * min(ts)
        grad = {"workload": "diff_8x160x120", "ms": gms, "edges": Ed, "passes": wd.iters, "loss": loss,
                "edge_updates_per_s": Ed * wd.iters / (gms / 1e3),
                "note": "forward passes with checkpoints, held-out loss and the reverse pass; synchronous call"}
        mp.close()

    # ---------------------------------------------------------------- CPU oracle on a bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        csr, ln = oracle_sample(w, 1)
        Es = int(csr["ray_off"][-1])
        t = run_oracle_timed(w, csr, ln, iters)
        cpu = {"value": Es * iters / t, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
               "sample": f"frame 0 of {args.workload} ({Es} edges), {iters} passes, full grid; {t:.1f} s"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": args.workload, "frames": len(w.frames),
                          "image": f"{w.frames[0].cam.W}x{w.frames[0].cam.H}",
                          "grid": f"{w.grid.nx}x{w.grid.ny}x{w.grid.nz}@{w.grid.res}", "passes": iters,
                          "prior": w.prior, "first_pass_message": w.init_p or w.prior,
                          "parallelism": "replicas" if world > 1 else "1gpu",
                          "l2": "inputs larger than L2 (per-edge arrays ~%.0f GB)" % (E * 16 / 1e9)},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(), "fp64_gpu": f64, "grad": grad, "variants": variants,
               "accuracy": {k: (v if k == "frame" else {"accurate": v[0], "evaluated": v[1],
                                                        "fraction": v[0] / max(v[1], 1)})
                            for k, v in acc.items()}, **extra}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
