"""Autotuner host logic: the choice rule, the workload signature and the
JSON cache (fake timings; no GPU)."""
import json
from dataclasses import dataclass

import pytest

from paper_1804_06231_gb300 import tune


def test_choose_picks_fastest_per_pass():
    calls = []

    def measure(d, b, td, tb, reps):
        calls.append((d, b, td, tb))
        return ({2: 5.0, 3: 4.0, 4: 3.0}[d] + {64: 0.5, 128: 0.2, 256: 0.1}[td],
                {1: 7.0, 2: 9.0, 3: 8.0}[b] + {64: 0.1, 128: 0.3, 256: 0.4}[tb])

    (d, b, td, tb), times = tune.choose(measure, reps=3)
    assert (d, b, td, tb) == (4, 1, 256, 64)
    assert times["density"] == {2: 5.2, 3: 4.2, 4: 3.2}
    assert times["backward"] == {1: 7.3, 2: 9.3, 3: 8.3}
    # CTAs: density shapes timed with the default backward shape and vice
    # versa, both at the default task block; then the task blocks at the
    # chosen CTAs
    assert all(b == tune.DEFAULT[1] and td == tb == tune.DEFAULT_TASK for d, b, td, tb in calls[:3])
    assert all(d == tune.DEFAULT[0] and td == tb == tune.DEFAULT_TASK for d, b, td, tb in calls[3:6])
    assert [c[2] for c in calls[6:]] == list(tune.TASK_CHOICES)
    assert all((c[0], c[1]) == (4, 1) and c[2] == c[3] for c in calls[6:])


def test_choose_prefers_default_on_ties():
    (d, b, td, tb), _ = tune.choose(lambda d, b, td, tb, r: (1.0, 1.0))
    assert (d, b) == tune.DEFAULT and td == tb == tune.DEFAULT_TASK
    # within the tie margin the default stays; beyond it the faster choice wins
    near = 1.0 / (1.0 + tune.TIE / 2)
    far = 1.0 / (1.0 + tune.TIE * 2)
    m = lambda d, b, td, tb, r: ({64: near, 128: 1.0, 256: 1.0}[td], {64: far, 128: 1.0, 256: 1.0}[tb])
    (_, _, td, tb), _ = tune.choose(m)
    assert td == tune.DEFAULT_TASK and tb == 64


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

    def set_tuning(self, d, b, td=None, tb=None):
        self.set.append((d, b, td, tb))


def test_autotune_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    g = _FakeGrid()
    n = {"calls": 0}

    def measure(d, b, td, tb, reps):
        n["calls"] += 1
        return {2: 2.0, 3: 1.0, 4: 1.5}[d], {1: 0.5, 2: 0.7, 3: 0.6}[b] + (0.2 if tb == 64 else 0.0)

    r1 = tune.autotune(g, None, cache_path=path, measure=measure, device_info=("GB300", 152))
    assert r1["source"] == "timed" and (r1["density_ctas_per_sm"], r1["backward_ctas_per_sm"]) == (3, 1)
    assert (r1["density_task_block"], r1["backward_task_block"]) == (128, 128)
    assert g.set[-1] == (3, 1, 128, 128) and n["calls"] == 9
    data = json.load(open(path))
    assert r1["signature"] in data
    r2 = tune.autotune(_FakeGrid(), None, cache_path=path, measure=measure,
                       device_info=("GB300", 152))
    assert r2["source"] == "cache" and n["calls"] == 9
    # another device: timed again, both entries kept
    tune.autotune(_FakeGrid(), None, cache_path=path, measure=measure, device_info=("B200", 148))
    assert len(json.load(open(path))) == 2 and n["calls"] == 18


def test_autotune_ignores_bad_cache(tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text("not json")
    r = tune.autotune(_FakeGrid(), None, cache_path=str(path),
                      measure=lambda d, b, td, tb, r: (1.0, 1.0), device_info=("GB300", 152))
    assert r["source"] == "timed"
    sig = r["signature"]
    path.write_text(json.dumps({sig: {"density_ctas_per_sm": 9, "backward_ctas_per_sm": 1,
                                      "density_task_block": 128, "backward_task_block": 128}}))
    r = tune.autotune(_FakeGrid(), None, cache_path=str(path),
                      measure=lambda d, b, td, tb, r: (1.0, 1.0), device_info=("GB300", 152))
    assert r["source"] == "timed"  # out-of-range entry is not used
    # an entry written before the task blocks were tuned is timed again
    path.write_text(json.dumps({sig: {"density_ctas_per_sm": 3, "backward_ctas_per_sm": 3}}))
    r = tune.autotune(_FakeGrid(), None, cache_path=str(path),
                      measure=lambda d, b, td, tb, r: (1.0, 1.0), device_info=("GB300", 152))
    assert r["source"] == "timed"
