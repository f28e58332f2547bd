"""The batch autotuner's search (host logic, no GPU): coordinate descent over
the launch shape and dedup cadence, timed here by a synthetic cost in place
of a batch run.  Every tuning gives the same results, so the search's only
job is to find a fast one: these tests check that it reaches the optimum of
a separable cost from the library's defaults, measures each configuration
once, keeps the incumbent unless a candidate is at least 2 % faster, stops
when a pass improves nothing, and remembers a workload's result by key."""
import json

import pytest

from paper_2108_05815_b300 import autotune


@pytest.fixture
def fake_timer(monkeypatch):
    """replaces the batch timing by cost(tuning); records every call"""
    calls = []

    def install(cost):
        def timed(make_sims, tuning, repeats):
            calls.append(dict(tuning))
            return cost(tuning)
        monkeypatch.setattr(autotune, "_time_batch", timed)
        return calls
    return install


# a separable cost with its optimum away from the defaults in every coordinate
BEST = {"block_threads": 512, "blocks_per_sm": 2, "lineages_per_lane": 4, "events_per_visit": 32,
        "occupancy_step": 0.5, "tail_events": 512.0, "coop_lineages": 4096}


def separable(t):
    cost = 1.0
    for k, want in BEST.items():
        vals = autotune.SPACE[k]
        # a default outside the candidates counts as beyond the last one
        at = vals.index(t[k]) if t[k] in vals else len(vals) + 1
        cost += 0.1 * abs(at - vals.index(want))
    return cost


def test_finds_the_optimum_of_a_separable_cost(fake_timer):
    calls = fake_timer(separable)
    best, secs, trials = autotune.tune(lambda: [], passes=3)
    assert {k: best[k] for k in BEST} == BEST
    assert secs == pytest.approx(1.0)
    # each configuration timed once (the search caches its measurements)
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys)) == trials


def test_keeps_the_defaults_when_nothing_is_two_percent_faster(fake_timer):
    defaults = {k: v for k, v in autotune.default_tuning().items() if k in autotune.SPACE}

    def flat(t):  # every other tuning 1.5 % faster: within the hysteresis
        return 1.0 if t == defaults else 0.985
    calls = fake_timer(flat)
    best, secs, trials = autotune.tune(lambda: [], passes=2)
    assert best == defaults and secs == 1.0
    # one pass over every coordinate, no second pass (nothing improved)
    assert trials == 1 + sum(len([v for v in vals if v != defaults[k]]) for k, vals in autotune.SPACE.items())
    assert len(calls) == trials


def test_one_coordinate_space(fake_timer):
    fake_timer(lambda t: {1: 3.0, 8: 2.0, 32: 1.0}[t["events_per_visit"]])
    best, secs, _ = autotune.tune(lambda: [], passes=1, space={"events_per_visit": [1, 8, 32]})
    assert best == {"events_per_visit": 32} and secs == 1.0


def test_cached_tune_remembers_by_key(fake_timer, tmp_path):
    calls = fake_timer(separable)
    path = str(tmp_path / "tuning.json")
    best, secs, trials = autotune.cached_tune("config4", lambda: [], path=path, passes=3)
    assert trials > 0 and {k: best[k] for k in BEST} == BEST
    n = len(calls)
    again, secs2, trials2 = autotune.cached_tune("config4", lambda: [], path=path, passes=3)
    assert again == best and secs2 == secs and trials2 == 0 and len(calls) == n
    assert json.load(open(path))["config4"]["tuning"] == best
