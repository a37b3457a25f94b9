"""The kernel-plan autotuner's host logic (timing replaced by a table): the fastest plan wins and is left
set, winners are stored per GPU name and configuration key, and applied only to a matching configuration."""
import json

import pytest

from paper_2006_03512_gb300 import autotune


class FakeMap:
    def __init__(self, n_rays, n_edges, max_len, n_scenes=1):
        self._st = {"n_rays": n_rays, "n_edges": n_edges, "max_ray_len": max_len}
        self.n_scenes = n_scenes
        self.plans = []

    def stats(self):
        return dict(self._st)

    def set_plan(self, *plan):
        self.plans.append(tuple(plan))


def test_config_key_buckets_by_powers_of_two():
    a = FakeMap(1000, 300_000, 478)
    assert autotune.config_key(a) == "maxlen512_mean512_E524288_single"
    b = FakeMap(1000, 290_000, 470)          # same buckets
    assert autotune.config_key(b) == autotune.config_key(a)
    c = FakeMap(1000, 300_000, 600, n_scenes=3)
    assert autotune.config_key(c) == "maxlen1024_mean512_E524288_batch"


def test_tune_stores_and_apply_reuses(monkeypatch, tmp_path):
    times = {(8, 256, 1): 5.0, (8, 256, 0): 7.0, (16, 128, 1): 4.0, (16, -1, 0): 9.0}
    monkeypatch.setattr(autotune, "time_plan", lambda mp, plan, iters, repeats=2: times[tuple(plan)])
    monkeypatch.setattr(autotune, "gpu_name", lambda: "FAKE GPU")
    path = str(tmp_path / "plans.json")
    mp = FakeMap(1000, 300_000, 478)
    entry = autotune.tune(mp, iters=2, path=path, candidates=list(times))
    assert entry["plan"] == [16, 128, 1] and entry["ms"] == 4.0
    assert mp.plans[-1] == (16, 128, 1)               # the winner is left set
    db = json.load(open(path))
    assert db["FAKE GPU"][autotune.config_key(mp)]["plan"] == [16, 128, 1]
    assert set(db["FAKE GPU"][autotune.config_key(mp)]["all_ms"]) == {"8,256,1", "8,256,0", "16,128,1", "16,-1,0"}
    # the same configuration elsewhere gets the stored plan without timing
    other = FakeMap(1000, 290_000, 470)
    monkeypatch.setattr(autotune, "time_plan", lambda *a, **k: pytest.fail("timed again"))
    assert autotune.apply(other, path) == (16, 128, 1) and other.plans == [(16, 128, 1)]
    # another configuration, or another GPU, has no entry
    assert autotune.apply(FakeMap(10, 300, 20), path) is None
    monkeypatch.setattr(autotune, "gpu_name", lambda: "OTHER GPU")
    assert autotune.apply(other, path) is None


def test_load_tolerates_a_missing_or_broken_file(tmp_path):
    assert autotune.load(str(tmp_path / "none.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert autotune.load(str(bad)) == {}


def test_committed_table_is_well_formed():
    db = autotune.load()
    assert db, "tuned_plans.json is committed"
    for gpu, entries in db.items():
        for key, e in entries.items():
            assert key.startswith("maxlen") and len(e["plan"]) == 3
            assert e["ms"] == min(e["all_ms"].values())
