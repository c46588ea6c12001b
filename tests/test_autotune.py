"""Autotuner search logic (CPU, with a synthetic cost surface) and, on the
GPU, that a tuned configuration gives the same results as the default."""
import numpy as np
import pytest

from paper_2202_13511_gb300 import autotune
from paper_2202_13511_gb300 import workloads as W


def test_coordinate_descent_finds_separable_minimum():
    space = {"a": [1, 2, 4, 8], "b": [0, 1], "c": [16, 64, 256]}
    target = {"a": 4, "b": 0, "c": 256}
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return sum((np.log2(cfg[k]) - np.log2(target[k])) ** 2 if k != "b" else (cfg[k] - target[k]) ** 2
                   for k in cfg) + 1.0

    best, t, hist = autotune.coordinate_descent({"a": 1, "b": 1, "c": 16}, space, measure)
    assert best == target and t == 1.0
    # every configuration is timed once
    assert len(calls) == len({tuple(sorted(c.items())) for c in calls}) == len(hist)


def test_coordinate_descent_keeps_start_on_ties():
    best, t, _ = autotune.coordinate_descent({"a": 2}, {"a": [1, 2, 3]}, lambda cfg: 5.0)
    assert best == {"a": 2} and t == 5.0


def test_confirm_best_times_the_leaders_again():
    """A configuration that was only lucky in the search loses the second
    timing of the leaders; the search history is what gets re-timed."""
    history = [({"a": 1}, 1.0), ({"a": 2}, 0.5), ({"a": 3}, 0.9), ({"a": 4}, 3.0)]
    again = {1: 0.95, 2: 1.2, 3: 0.85, 4: 0.1}  # a = 4 was not among the three leaders
    seen = []

    def measure(cfg):
        seen.append(cfg["a"])
        return again[cfg["a"]]

    best, t = autotune.confirm_best(history, measure)
    assert best == {"a": 3} and t == 0.85
    assert sorted(seen) == [1, 2, 3]


def test_tune_server_confirms_with_its_timer():
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return 1.0 + abs(cfg["slots"] - 2) + (0 if cfg["max_batch"] == 64 else 0.5)

    best, t, hist = autotune.tune_server([], measure=measure)
    assert best == {"slots": 2, "max_batch": 64} and t == 1.0
    assert len(calls) == len(hist) + 3  # the search, then the three leaders again


def test_relevant_space_drops_block_knobs_for_trees():
    trees = [W.snowflake(10, seed=s) for s in range(3)]
    assert set(autotune.relevant_space(trees)) == {"grid_blocks_per_sm", "filter", "lanes",
                                                   "group_threads_log2"}
    mixed = trees + [W.cyclic(10, seed=1)]
    assert set(autotune.relevant_space(mixed)) == set(autotune.KERNEL_SPACE)
    cycles = [W.cyclic(10, seed=s) for s in range(2)]
    assert set(autotune.relevant_space(cycles)) == set(autotune.KERNEL_SPACE) - {"group_threads_log2"}


def test_tune_kernels_with_injected_timer():
    qs = [W.cyclic(12, seed=s) for s in range(2)]
    best, t, hist = autotune.tune_kernels(
        qs, measure=lambda cfg: 1.0 + abs(cfg["grid_blocks_per_sm"] - 4) + cfg["use_ccc"] * 0.5)
    assert best["grid_blocks_per_sm"] == 4 and best["use_ccc"] == 0


@pytest.mark.gpu
def test_tuned_config_same_results():
    from paper_2202_13511_gb300 import mpdp
    qs = [W.snowflake(18, seed=s) for s in range(8)] + [W.cyclic(15, seed=s) for s in range(8)]
    best, t, hist = autotune.tune_kernels(qs, reps=1)
    assert t > 0 and len(hist) >= 3
    with mpdp.Optimizer(0) as o:
        ref = [(p.cost, p.signature()) for p in o.optimize_batch(qs)]
        o.set_config(**best)
        got = [(p.cost, p.signature()) for p in o.optimize_batch(qs)]
    assert [np.float64(c).tobytes() for c, _ in got] == [np.float64(c).tobytes() for c, _ in ref]
    assert [s for _, s in got] == [s for _, s in ref]
