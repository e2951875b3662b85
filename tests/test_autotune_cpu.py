"""CPU checks of the autotuner's search and cache (a fake plan and timer: no GPU)."""
import json

import pytest

from paper_2501_05244_gb300 import autotune as at
from paper_2501_05244_gb300.nursd import NursdError


class FakePlan:
    N, F, Z, T = 128, 64, 64, 512

    def __init__(self):
        self.values = {"batch_grouped": 1, "spread_rows": 8, "batch_streams": 4}

    def tune(self, name, value):
        if name == "spread_rows" and value not in (4, 8, 16):
            raise NursdError(5, "nursd_plan_tune")
        self.values[name] = value

    def tuning(self):
        return dict(self.values)


def fake_timer(plan, cost):
    # the "time" of a step is a fixed function of the plan's current settings
    return lambda step, reps, warmup: cost(plan.values)


def test_coordinate_descent_picks_the_fastest_setting_and_caches_it(tmp_path):
    plan = FakePlan()
    cost = lambda v: abs(v["spread_rows"] - 16) + abs(v["batch_streams"] - 2) * 3 + (1 - v["batch_grouped"]) * 5 + 1.0
    path = str(tmp_path / "tune.json")
    r = at.autotune(plan, lambda: None, workload="B=64", cache_path=path, timer=fake_timer(plan, cost), gpu="GB300")
    assert r["choice"] == {"batch_grouped": 1, "spread_rows": 16, "batch_streams": 2} and not r["cached"]
    assert plan.values == r["choice"] and r["ms"] == 1.0
    assert len(r["results"]) == 2 + 3 + 5
    stored = json.load(open(path))
    assert r["key"] in stored and stored[r["key"]]["choice"] == r["choice"]
    # a second plan of the same key takes the cached choice without timing
    plan2 = FakePlan()
    never = lambda step, reps, warmup: pytest.fail("a cached choice must not be timed")
    r2 = at.autotune(plan2, lambda: None, workload="B=64", cache_path=path, timer=never, gpu="GB300")
    assert r2["cached"] and plan2.values == r["choice"]
    # another GPU or workload is another key
    assert at.shape_key(plan, "B=64", gpu="GB300") != at.shape_key(plan, "B=32", gpu="GB300")
    assert at.shape_key(plan, "B=64", gpu="GB300") != at.shape_key(plan, "B=64", gpu="B200")


def test_inapplicable_values_are_skipped(tmp_path):
    plan = FakePlan()
    r = at.autotune(plan, lambda: None, space={"spread_rows": (3, 8, 32)}, cache_path=str(tmp_path / "t.json"),
                    timer=fake_timer(plan, lambda v: 1.0), gpu="x")
    assert r["results"] == {"spread_rows=8": 1.0} and r["choice"] == {"spread_rows": 8}
