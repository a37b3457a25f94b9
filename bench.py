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
# implementation overhead of the (tile, voxel) groups, reported apart from the
# method's bytes: the ray kernel also reads each edge's window index (u16) and
# the ray-start and group-end bitmaps, and writes one partial sum per group;
# the voxel totals then read a slot index and gather a partial per group
BYTES_GROUP_EDGE = 2.25
BYTES_GROUP_PARTIAL = 4
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


def lib_init_p(w):
    """The first-pass message as the library receives it (mrf_options.init_p is a float)."""
    return float(np.float32(w.init_p or w.prior))


def run_oracle_timed(w, csr, ln, iters, init_p=None):
    """The oracle's BP on its sample: (seconds, marginals)."""
    import oracle
    t0 = time.perf_counter()
    p = oracle.bp(csr["ray_off"], csr["vox"], ln, w.grid.n_voxels, w.prior,
                  lib_init_p(w) if init_p is None else init_p, oracle.default_log_nu_bg(w.lut), iters)[2]
    return time.perf_counter() - t0, p


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
    ts = [run_oracle_timed(w, csr, ln, args.iters or w.iters)[0] for _ in range(args.steps)]
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


def batch_waves(n_scenes):
    """Scenes 0..n-1 of the 64-scene batch cut into waves of about 2.5e9 edges (estimated as frames x
    pixels x grid edge): the collection exceeds one context's 2^32-edge index and the device memory."""
    from synth.scenes import batch_scene_size
    waves, cur, tot = [], [], 0
    for i in range(n_scenes):
        n, nf = batch_scene_size(i)
        est = nf * 320 * 240 * n
        if cur and tot + est > 2.5e9:
            waves.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += est
    waves.append(cur)
    return waves


def generate_batch_scenes(indices):
    """Renders batch scenes on the host cores (a spawn pool, safe whether or not CUDA is up)."""
    import concurrent.futures as cf
    import multiprocessing as mpr
    with cf.ProcessPoolExecutor(max_workers=os.cpu_count() or 4, mp_context=mpr.get_context("spawn")) as ex:
        return dict(ex.map(_batch_scene, indices))


def ray_roofline(E, G, S, iters, steps, prof, peak, peak_kind, traffic_per_edge=None):
    """Roofline of the ray kernel and the voxel totals from their CUDA-event times over `steps` calls of
    mrf_infer(iters): the method's bytes (20 B/edge, 8 on the first pass; voxel totals 8 B per
    partial read + 12 B per voxel) over the measured time; the grouping's extra bytes beside them."""
    ray_bytes = E * (BYTES_RAY_EDGE_FIRST + BYTES_RAY_EDGE * (iters - 1)) * steps
    ray_overhead = (E * BYTES_GROUP_EDGE + G * BYTES_GROUP_PARTIAL) * iters * steps if G > 0 else 0.0
    if G > 0:
        red_bytes = (G * BYTES_RED_GROUP + S * BYTES_RED_SEG) * iters * steps
    else:
        red_bytes = (E * BYTES_RED_EDGE + S * BYTES_RED_SEG) * iters * steps
    ray_gbs = ray_bytes / (prof["ms_ray_messages"] / 1e3) / 1e9
    red_gbs = red_bytes / (prof["ms_voxel_reduce"] / 1e3) / 1e9
    n_ray, n_red = prof["n_ray_messages"], prof["n_voxel_reduce"]
    if prof["ms_ray_messages"] >= prof["ms_voxel_reduce"]:
        dom, ach, nl, byt, ovh = "ray_messages", ray_gbs, n_ray, ray_bytes, ray_overhead
    else:
        dom, ach, nl, byt, ovh = "voxel_reduce", red_gbs, n_red, red_bytes, 0.0
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_kind": peak_kind,
            "traffic": traffic_per_edge * E if traffic_per_edge else None,
            "algorithmic_bytes_per_launch": byt / max(nl, 1),
            "overhead_bytes_per_launch": ovh / max(nl, 1),
            "overhead": "(tile, voxel) grouping: window index 2 B + bitmaps 0.25 B per edge, 4 B per group partial",
            "launches": nl,
            "other_kernel": {"ray_messages": {"GB/s": ray_gbs, "ms": prof["ms_ray_messages"]},
                             "voxel_reduce": {"GB/s": red_gbs, "ms": prof["ms_voxel_reduce"]},
                             "other_ms": prof["ms_other_infer"]}}


def oracle_errors(torch, m, w, iters, stream, p_ref, sens):
    """Whole-BP marginals of the GPU's FP32 and FP64 forms on the oracle's sample (the first frame of
    the workload, full grid, same passes) against the oracle's: max, count above 1e-4, and the same on
    the voxels the oracle's own rounding-size probe moves by at most 5e-6 (well-conditioned)."""
    fr = w.frames[0]
    well = sens <= 5e-6
    out = {"sample": "frame 0, full grid, %d passes" % iters, "sensitive_voxels": int((~well).sum()),
           "probe": "FP64 oracle with 1e-7 relative noise on its likelihoods, and with its first-pass log-odds "
                    "one float32 ulp up; sensitive: either moves p by > 5e-6",
           "first_pass_message": "as the library receives it (float32)"}
    for name, prec in (("fp32", m.PREC_F32), ("fp64", m.PREC_F64)):
        mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p, precision=prec), stream=stream)
        mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
        mp.infer(iters)
        if prec == m.PREC_F64:
            _, T = mp.export_messages()
            p = (1.0 / (1.0 + torch.exp(-T.double()))).cpu().numpy()
        else:
            p = mp.marginals().double().cpu().numpy().ravel()
        mp.close()
        err = np.abs(p - p_ref)
        out[name] = {"max": float(err.max()), "n_above_1e-4": int((err > 1e-4).sum()),
                     "max_well_conditioned": float(err[well].max()) if well.any() else 0.0,
                     "n_above_1e-4_well_conditioned": int((err[well] > 1e-4).sum())}
    return out


class Runner:
    """One workload on this GPU: device-resident timing of mrf_infer, its roofline, and end to end
    through the C ABI with host buffers."""

    def __init__(self, torch, m, stream, sync, dist, world, plan=None):
        self.torch, self.m, self.stream, self.sync, self.dist, self.world, self.plan = \
            torch, m, stream, sync, dist, world, plan

    def device(self, w, iters, steps, warmup, clocks=None):
        torch, m, stream = self.torch, self.m, self.stream
        depths = [torch.from_numpy(fr.depth).cuda() for fr in w.frames]
        mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p), stream=stream)
        if self.plan:
            mp.set_plan(*self.plan)
        mp.profile(True)
        for d, fr in zip(depths, w.frames):
            mp.add_frame(d, fr.cam.pose, fr.cam, w.lut)
        mp.infer(iters)            # first call builds the transpose
        mp.synchronize()
        prof0 = mp.profile_read()
        st = mp.stats()
        for _ in range(max(warmup - 1, 0)):
            mp.infer(iters)
        mp.profile_read()
        self.sync()
        launches0 = mp.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with (ClockSampler(torch.cuda.current_device()) if clocks is None else clocks) as clk:
            self.sync()
            ev0.record(stream)
            for _ in range(steps):
                mp.infer(iters)
            ev1.record(stream)
            self.sync()
        return {"mp": mp, "depths": depths, "ms": ev0.elapsed_time(ev1), "prof0": prof0,
                "prof": mp.profile_read(), "stats": st, "launches": mp.launch_count() - launches0,
                "clocks": clk.summary() if clocks is None else None, "plan": mp.plan_info()}

    def e2e(self, w, iters, steps):
        torch, m = self.torch, self.m
        pinned = [torch.from_numpy(fr.depth).pin_memory().numpy() for fr in w.frames]
        out = torch.empty(w.grid.n_voxels, dtype=torch.float32).pin_memory().numpy()
        mp = m.Map(w.grid, w.prior, m.Options(init_p=w.init_p), stream=self.stream)
        if self.plan:
            mp.set_plan(*self.plan)

        def step():
            mp.reset()
            for d, fr in zip(pinned, w.frames):
                mp.add_frame(d, fr.cam.pose, fr.cam, w.lut)
            mp.infer(iters)
            mp.marginals_host(out.reshape(mp.shape))

        step()
        self.sync()
        k = max(1, min(steps, 3))
        t0 = time.perf_counter()
        for _ in range(k):
            step()
        self.sync()
        dt = _barrier_max(torch, self.dist, self.world, (time.perf_counter() - t0) / k)
        E = mp.stats()["n_edges"]
        mp.close()
        return {"value": _sum(torch, self.dist, self.world, float(E) * iters) / dt, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(fr.depth.nbytes for fr in w.frames)),
                "d2h_bytes_per_step": int(w.grid.n_voxels * 4), "ms_per_step": dt * 1e3, "steps": k}


def corridor_leg(torch, m, stream, sync, args, peak, peak_kind):
    """The scale workload (60 frames of 424x240 along a corridor into a room, 512x512x256, 30
    passes): value, roofline and e2e as for the room, and the frame-0 comparison with the oracle."""
    from synth import make_workload
    w = make_workload("corridor_60x424x240")
    iters = w.iters
    steps = max(1, min(args.steps, 3))
    r = Runner(torch, m, stream, sync, None, 1)
    d = r.device(w, iters, steps, 2)
    E, st, prof = d["stats"]["n_edges"], d["stats"], d["prof"]
    G, S = d["plan"]["n_groups"], st["n_touched"]
    d["mp"].close()
    del d["depths"]
    out = {"workload": "corridor_60x424x240", "value": E * iters * steps / (d["ms"] / 1e3), "unit": UNIT,
           "ms_per_step": d["ms"] / steps, "steps": steps, "passes": iters, "edges": E,
           "max_ray_len": st["max_ray_len"], "groups": G,
           "roofline": ray_roofline(E, G, S, iters, steps, prof, peak, peak_kind),
           "gpu_launches": d["launches"], "clocks": d["clocks"],
           "l2": "inputs larger than L2 (per-edge arrays ~%.0f GB)" % (E * 16 / 1e9)}
    out["e2e"] = r.e2e(w, iters, steps)
    if not args.no_cpu:
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        csr, ln = oracle_sample(w, 1)
        t, p_ref = run_oracle_timed(w, csr, ln, iters)
        sens = oracle_probe(w, csr, ln, iters, p_ref)
        out["errors_vs_oracle"] = oracle_errors(torch, m, w, iters, stream, p_ref, sens)
    return out


def batch_leg(torch, m, stream, args, peak, peak_kind, n_waves=2):
    """A bounded part of the 64-scene batch (uneven grids 64^3-192^3 at 0.03 m, 8-60 frames of
    320x240, 15 passes): its first waves, each a batched context whose passes replay as one CUDA
    graph (value); one profiled mrf_infer per wave (roofline); and end to end per wave from pinned
    host frames through the C ABI (e2e)."""
    from paper_2006_03512_gb300 import autotune
    waves = batch_waves(64)[:n_waves]
    idx = [i for wv in waves for i in wv]
    t0 = time.perf_counter()
    scenes = generate_batch_scenes(idx)
    gen_s = time.perf_counter() - t0
    iters = scenes[idx[0]].iters
    steps = max(1, min(args.steps, 3))
    E_all, G_all, S_all, ms_all, e2e_s, plans = 0, 0, 0, 0.0, 0.0, []
    prof_all = {"ms_ray_messages": 0.0, "ms_voxel_reduce": 0.0, "ms_other_infer": 0.0, "n_ray_messages": 0,
                "n_voxel_reduce": 0}
    h2d, d2h = 0, 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for wv in waves:
            ws = [scenes[i] for i in wv]
            mp = m.Map([w.grid for w in ws], 0.5, m.Options(init_p=ws[0].init_p), stream=stream)
            for s, w in enumerate(ws):
                for fr in w.frames:
                    mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut, scene=s)
            plan = autotune.apply(mp)
            if plan is None:
                plan = tuple(autotune.tune(mp, iters=3)["plan"])
            plans.append(list(plan))
            mp.infer(1)                 # builds the transpose
            mp.infer_graph(iters)       # records
            mp.infer_graph(iters)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                mp.infer_graph(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_all += e0.elapsed_time(e1) / steps
            mp.profile(True)
            mp.profile_read()
            mp.infer(iters)
            pr = mp.profile_read()
            for k in prof_all:
                prof_all[k] += pr[k]
            E_all += mp.stats()["n_edges"]
            G_all += mp.plan_info()["n_groups"]
            S_all += mp.stats()["n_touched"]
            nv = mp.n_voxels
            mp.close()
            # end to end: the wave's frames from pinned host memory, build, passes, marginals back
            pinned = [[torch.from_numpy(fr.depth).pin_memory() for fr in w.frames] for w in ws]
            outp = torch.empty(nv, dtype=torch.float32).pin_memory().numpy()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            mp = m.Map([w.grid for w in ws], 0.5, m.Options(init_p=ws[0].init_p), stream=stream)
            mp.set_plan(*plan)
            for s, w in enumerate(ws):
                for d, fr in zip(pinned[s], w.frames):
                    # batched contexts take device frames: copy each from pinned host memory
                    mp.add_frame(d.cuda(non_blocking=True), fr.cam.pose, fr.cam, w.lut, scene=s)
            mp.infer(iters)
            mp.marginals_host(outp)
            torch.cuda.synchronize()
            e2e_s += time.perf_counter() - t1
            h2d += sum(fr.depth.nbytes for w in ws for fr in w.frames)
            d2h += nv * 4
            mp.close()
    return {"workload": "batch64 (first %d waves)" % len(waves), "scenes": idx, "waves": len(waves),
            "value": E_all * iters / (ms_all / 1e3), "unit": UNIT, "ms_per_step": ms_all, "steps": steps,
            "passes": iters, "edges": E_all, "plans": plans, "graph": True,
            "roofline": ray_roofline(E_all, G_all, S_all, iters, 1, prof_all, peak, peak_kind),
            "e2e": {"value": E_all * iters / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "note": "per wave: a new batched context, frames from pinned host memory, build, passes, "
                            "marginals back; waves in sequence"},
            "generate_s": gen_s, "clocks": clk.summary(),
            "l2": "inputs larger than L2 (per-edge arrays of every wave > 10 GB)"}


def batch_bench(args):
    """The whole 64-scene batch, all waves (bench.py --workload batch64)."""
    rank, world, local = _dist()
    if rank != 0:
        return 0
    import torch
    import paper_2006_03512_gb300 as m
    m.build()
    torch.cuda.set_device(local)
    peak, peak_kind = _peaks()
    leg = batch_leg(torch, m, torch.cuda.current_stream(), args, peak, peak_kind, n_waves=10 ** 6)
    out = {"metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": 1, "steps": leg["steps"],
           "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch64", "waves": leg["waves"], "passes": leg["passes"],
                      "edges": leg["edges"], "plans": leg["plans"], "graph": True, "l2": leg["l2"]},
           "roofline": leg["roofline"], "e2e": leg["e2e"], "clocks": leg["clocks"],
           "gpu_launches": None, "generate_s": leg["generate_s"]}
    print(json.dumps(out))
    return 0


def oracle_probe(w, csr, ln, iters, p_ref):
    """|dp| per voxel of the oracle under rounding-size changes of the inputs FP32 must round: 1e-7
    relative noise on its likelihoods, and its first-pass log-odds moved by one float32 ulp (every
    edge at once); the larger of the two."""
    import oracle
    rng = np.random.default_rng(0)
    ip = lib_init_p(w)
    lbg = oracle.default_log_nu_bg(w.lut)
    p1 = oracle.bp(csr["ray_off"], csr["vox"], ln + rng.normal(0, 1e-7, len(ln)), w.grid.n_voxels, w.prior,
                   ip, lbg, iters)[2]
    d = np.abs(p1 - p_ref)
    L0 = np.log(ip) - np.log1p(-ip)
    if L0 != 0:
        ip1 = float(1.0 / (1.0 + np.exp(-(L0 + float(np.spacing(np.float32(abs(L0))))))))
        p2 = oracle.bp(csr["ray_off"], csr["vox"], ln, w.grid.n_voxels, w.prior, ip1, lbg, iters)[2]
        d = np.maximum(d, np.abs(p2 - p_ref))
    return d


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
    ap.add_argument("--no-legs", action="store_true", help="skip the corridor and batch legs")
    ap.add_argument("--e2e-only", action="store_true",
                    help="time only the end-to-end steps (for launch lists of them; not a bench line)")
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

    plan = tuple(int(x) for x in args.plan.split(",")) if args.plan else None
    runner = Runner(torch, m, stream, sync, dist, world, plan)
    if args.e2e_only:
        e2e = runner.e2e(w, iters, args.steps)
        if rank == 0:
            print(json.dumps({"workload": args.workload, "e2e": e2e}))
        return
    opts = dict(init_p=w.init_p)

    # ---------------------------------------------------------------- device-resident run
    if args.steps == 0:   # set-up only (profiling runs that capture the first passes)
        d = runner.device(w, iters, 0, args.warmup)
        d["mp"].close()
        return 0
    d = runner.device(w, iters, args.steps, args.warmup)
    mp, depths, st, prof, prof0 = d["mp"], d["depths"], d["stats"], d["prof"], d["prof0"]
    E, S = st["n_edges"], st["n_touched"]
    ms = d["ms"]
    ms_max = _barrier_max(torch, dist, world, ms)
    edge_updates = _sum(torch, dist, world, float(E) * iters * args.steps)
    value = edge_updates / (ms_max / 1e3)

    # roofline of the dominant kernel (times from the same timed region)
    peak, peak_kind = _peaks()
    G = d["plan"]["n_groups"]
    key = "ray_messages_f32" if prof["ms_ray_messages"] >= prof["ms_voxel_reduce"] else "voxel_reduce_f32"
    tr = _ncu_traffic(key)
    roofline = ray_roofline(E, G, S, iters, args.steps, prof, peak, peak_kind,
                            tr["bytes_per_edge"] if tr else None)
    model_frac = (28.0 * E * iters * args.steps / (ms / 1e3) / 1e9) / peak

    # traversal and transpose throughput (from the first build above)
    extra = {"edges": E, "rays": st["n_rays"], "touched_voxels": S, "max_ray_len": st["max_ray_len"],
             "groups": G,
             "traverse_edges_per_s": E / (prof0["ms_traverse"] / 1e3) if prof0["ms_traverse"] else None,
             "transpose_ms": prof0["ms_build"], "whole_step_model_frac": model_frac}
    p32 = mp.marginals().clone()   # for the error against the FP64 form
    extra["plan"] = d["plan"]
    # the paper's accuracy metric of the map on its first frame
    fr0 = w.frames[0]
    acc = {"frame": 0, "fp32": mp.accuracy(depths[0], fr0.cam.pose, fr0.cam, w.lut)}
    mp.close()
    launches, clocks_room = d["launches"], d["clocks"]
    del depths, d

    # ---------------------------------------------------------------- end to end through the C ABI
    e2e = None if args.no_e2e else runner.e2e(w, iters, args.steps)

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
        # ablation: the paper's log-domain message form in FP32 (Kahan-compensated log P), timed the same way
        mp = m.Map(w.grid, w.prior, m.Options(precision=m.PREC_F32_LOG, **opts), stream=stream)
        for fr in w.frames:
            mp.add_frame(torch.from_numpy(fr.depth).cuda(), fr.cam.pose, fr.cam, w.lut)
        mp.infer(iters)
        sync()
        e0.record(stream)
        mp.infer(iters)
        e1.record(stream)
        sync()
        gms = e0.elapsed_time(e1)
        f64["errors_vs_fp64"]["fp32_log_domain"] = _err_summary(torch, mp.marginals(), p64)
        f64["fp32_log_domain"] = {"value": float(E) * iters / (gms / 1e3), "unit": UNIT, "ms_per_step": gms,
                                  "form": "Eqs. pos/neg in the log domain, FP32, Kahan-compensated log P, "
                                          "thread per ray, per-edge voxel totals"}
        mp.close()
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
    cpu, errs = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        csr, ln = oracle_sample(w, 1)
        Es = int(csr["ray_off"][-1])
        t, p_ref = run_oracle_timed(w, csr, ln, iters)
        cpu = {"value": Es * iters / t, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
               "sample": f"frame 0 of {args.workload} ({Es} edges), {iters} passes, full grid; {t:.1f} s"}
        # the oracle's marginals on that sample against the GPU's FP32 and FP64 forms, voxel by voxel
        errs = oracle_errors(torch, m, w, iters, stream, p_ref, oracle_probe(w, csr, ln, iters, p_ref))
        del csr, ln, p_ref

    # ---------------------------------------------------------------- the scale workload and the batch
    legs = {}
    if rank == 0 and world == 1 and not args.no_legs and args.workload == WORKLOAD and not args.frames:
        legs["corridor"] = corridor_leg(torch, m, stream, sync, args, peak, peak_kind)
        legs["batch"] = batch_leg(torch, m, stream, args, peak, peak_kind)

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
               "clocks": clocks_room, "errors_vs_oracle": errs, "fp64_gpu": f64, "grad": grad,
               "variants": variants,
               "accuracy": {k: (v if k == "frame" else {"accurate": v[0], "evaluated": v[1],
                                                        "fraction": v[0] / max(v[1], 1)})
                            for k, v in acc.items()}, **legs, **extra}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
