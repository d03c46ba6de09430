"""Autotuner host logic: the choice rule, the workload signature and the
JSON cache (fake timings; no GPU)."""
import json
from dataclasses import dataclass

import pytest

from paper_1804_06231_gb300 import tune


def test_choose_picks_fastest_per_pass():
    calls = []

    def measure(d, b, reps):
        calls.append((d, b))
        return {2: 5.0, 3: 4.0, 4: 3.0}[d], {1: 7.0, 2: 9.0, 3: 8.0}[b]

    (d, b), times = tune.choose(measure, reps=3)
    assert (d, b) == (4, 1)
    assert times["density"] == {2: 5.0, 3: 4.0, 4: 3.0}
    assert times["backward"] == {1: 7.0, 2: 9.0, 3: 8.0}
    # density shapes are timed with the default backward shape and vice versa
    assert all(b == tune.DEFAULT[1] for d, b in calls[:3])
    assert all(d == tune.DEFAULT[0] for d, b in calls[3:])


def test_choose_prefers_default_on_ties():
    (d, b), _ = tune.choose(lambda d, b, r: (1.0, 1.0))
    assert (d, b) == tune.DEFAULT


def test_signature_buckets():
    s1 = tune.signature(1 << 20, 3375, 369, 1, "GB300", 152)
    s2 = tune.signature((1 << 20) + 5000, 3375, 400, 1, "GB300", 152)
    s3 = tune.signature(1 << 22, 68921, 21392, 1, "GB300", 152)
    assert s1 == s2 and s1 != s3
    assert "mean8" in s1 and "max8" in s1 and "n20" in s1
    assert tune.signature(0, 0, 0, 1, "x", 1).endswith("n0|mean0|max0")


@dataclass
class _Stats:
    n_particles: int = 100000
    n_cells: int = 1000
    max_cell_count: int = 300


class _FakeGrid:
    n = 100000
    boxes = [(0, 100000, 1.0, 10)]

    def __init__(self):
        self.set = []

    def stats(self):
        return _Stats()

    def set_tuning(self, d, b):
        self.set.append((d, b))


def test_autotune_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    g = _FakeGrid()
    n = {"calls": 0}

    def measure(d, b, reps):
        n["calls"] += 1
        return {2: 2.0, 3: 1.0, 4: 1.5}[d], {1: 0.5, 2: 0.7, 3: 0.6}[b]

    r1 = tune.autotune(g, None, cache_path=path, measure=measure, device_info=("GB300", 152))
    assert r1["source"] == "timed" and (r1["density_ctas_per_sm"], r1["backward_ctas_per_sm"]) == (3, 1)
    assert g.set[-1] == (3, 1) and n["calls"] == 6
    data = json.load(open(path))
    assert r1["signature"] in data
    r2 = tune.autotune(_FakeGrid(), None, cache_path=path, measure=measure,
                       device_info=("GB300", 152))
    assert r2["source"] == "cache" and n["calls"] == 6
    # another device: timed again, both entries kept
    tune.autotune(_FakeGrid(), None, cache_path=path, measure=measure, device_info=("B200", 148))
    assert len(json.load(open(path))) == 2 and n["calls"] == 12


def test_autotune_ignores_bad_cache(tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text("not json")
    r = tune.autotune(_FakeGrid(), None, cache_path=str(path), measure=lambda d, b, r: (1.0, 1.0),
                      device_info=("GB300", 152))
    assert r["source"] == "timed"
    sig = r["signature"]
    path.write_text(json.dumps({sig: {"density_ctas_per_sm": 9, "backward_ctas_per_sm": 1}}))
    r = tune.autotune(_FakeGrid(), None, cache_path=str(path), measure=lambda d, b, r: (1.0, 1.0),
                      device_info=("GB300", 152))
    assert r["source"] == "timed"  # out-of-range entry is not used
