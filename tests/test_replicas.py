"""The N-GPU bench path (replicas: one independent map per rank, no data-path collective) on CPU ranks.

What the replica runs share is the reduction of their timings and counts: the slowest rank's time and
the sum of the ranks' edge updates, and only rank 0 prints.  These run here as two gloo ranks on the host.
"""
import importlib.util
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    r, w, local = b._dist()
    ms = [12.5, 20.0][rank]          # per-rank timed region
    edges = [3.0e9, 5.0e9][rank]     # per-rank edge updates
    res = {"rank": r, "world": w, "local": local,
           "max_ms": b._barrier_max(torch, dist, w, ms), "sum_edges": b._sum(torch, dist, w, edges)}
    # the reference arm: ranks other than 0 leave without work
    class A:
        steps, warmup, iters, gpus = 1, 0, 1, world
    if rank != 0:
        res["reference_rc"] = b.reference_arm(A())
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r, x in enumerate(res):
        assert (x["rank"], x["world"], x["local"]) == (r, 2, r)
        assert x["max_ms"] == 20.0                       # the slowest rank's time, on every rank
        assert x["sum_edges"] == 8.0e9                   # whole-job work, on every rank
    assert res[1]["reference_rc"] == 0
    # whole-job throughput as the bench forms it: all ranks' work over the slowest rank's time
    assert res[0]["sum_edges"] / (res[0]["max_ms"] / 1e3) == pytest.approx(4.0e11)
