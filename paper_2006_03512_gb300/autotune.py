"""Kernel-plan autotuner: times candidate plans on a map and keeps the fastest per (GPU, configuration).

A plan is (edges per ray-kernel thread, threads per CTA or -1 for the tile-per-CTA kernel, per-(tile,
voxel) partial sums on/off) as set by ``Map.set_plan`` (mrf_set_plan).  The configuration key buckets
what decides the winner: the longest ray, the mean ray length, the edge count and whether the context
holds several scenes.  Winners are stored in a JSON file, keyed by the GPU's name and then the
configuration key, so a later run on the same kind of GPU and input applies them without timing.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

Plan = Tuple[int, int, int]

# every plan the library accepts for rays up to its longest supported length; plans a map's rays do
# not allow fall back to the library's choice inside the library, and are timed as such
CANDIDATES: List[Plan] = [
    (8, 256, 1), (8, 256, 0), (16, 256, 1), (16, 128, 1), (16, 128, 0), (4, 512, 1),
    (8, -1, 0), (16, -1, 0), (32, -1, 0),
]

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_plans.json")


def config_key(mp) -> str:
    """Bucketed description of a map's rays: longest ray and mean ray length (powers of two), edge
    count (power of two) and batching."""
    st = mp.stats()
    n_rays_hit = max(1, st["n_rays"])
    mean = st["n_edges"] / n_rays_hit
    b = lambda x: 1 << max(0, math.ceil(math.log2(max(1.0, x))))
    return f"maxlen{b(st['max_ray_len'])}_mean{b(mean)}_E{b(st['n_edges'])}_{'batch' if mp.n_scenes > 1 else 'single'}"


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def time_plan(mp, plan: Plan, iters: int, repeats: int = 2) -> float:
    """Milliseconds of `iters` passes under `plan` (the build happens in an untimed warm-up)."""
    import torch
    mp.set_plan(*plan)
    mp.infer(1)
    best = math.inf
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        mp.infer(iters)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def load(path: str = DEFAULT_PATH) -> Dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(mp, iters: int = 3, path: Optional[str] = DEFAULT_PATH,
         candidates: Sequence[Plan] = CANDIDATES) -> Dict:
    """Time every candidate on `mp`, leave the fastest set on it, and (with a path) record it."""
    times = {}
    for plan in candidates:
        times[",".join(map(str, plan))] = time_plan(mp, plan, iters)
    best = min(times, key=times.get)
    plan = tuple(int(x) for x in best.split(","))
    mp.set_plan(*plan)
    entry = {"plan": list(plan), "ms": times[best], "iters": iters, "all_ms": times}
    if path:
        db = load(path)
        db.setdefault(gpu_name(), {})[config_key(mp)] = entry
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return entry


def apply(mp, path: str = DEFAULT_PATH) -> Optional[Plan]:
    """Set the recorded plan for this GPU and the map's configuration, if there is one."""
    entry = load(path).get(gpu_name(), {}).get(config_key(mp))
    if not entry:
        return None
    plan = tuple(int(x) for x in entry["plan"])
    mp.set_plan(*plan)
    return plan
