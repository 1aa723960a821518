"""Host logic of the planner studies: the scenario sampler, the 2 % convergence rule and
the asset groups of the plan vector."""
import numpy as np

from paper_2410_13055_gb300 import study, synth


def test_batches_are_distinct_and_uniform():
    S, B = 16, 4
    draw = study.batches(S, B, seed=3)
    counts = np.zeros(S)
    for _ in range(4000):
        idx = next(draw)
        assert idx.size == B and np.unique(idx).size == B and idx.min() >= 0 and idx.max() < S
        assert np.all(np.diff(idx) > 0)
        counts[idx] += 1
    freq = counts / counts.sum()
    # uniform sampling without replacement: every scenario in B/S of the batches
    assert np.max(np.abs(freq - 1.0 / S)) < 0.01
    assert next(study.batches(3, 8, 0)).size == 3  # batch larger than the set: the whole set


def test_within_two_percent_rule():
    hist = [(0, 200.0), (5, 130.0), (10, 103.0), (15, 101.5), (20, 100.0)]
    assert study.within(hist, 100.0) == 15          # 101.5 <= 102
    assert study.within(hist, 100.0, rel=0.05) == 10
    assert study.within(hist, 50.0) is None
    neg = [(0, -90.0), (5, -97.0), (10, -98.5), (15, -100.0)]
    assert study.within(neg, -100.0) == 10           # -98.5 <= -100 + 2, -97 is not


def test_within_gap_rule():
    hist = [(0, 200.0), (5, 130.0), (10, 103.0), (15, 101.5), (20, 100.0)]
    # gap 100: within 2 of the target
    assert study.within_gap(hist, 200.0, 100.0) == 15
    assert study.within_gap(hist, 200.0, 100.0, frac=0.05) == 10
    assert study.within_gap(hist, 200.0, 97.0) is None  # needs J <= 99.06
    # a warm history measured against the cold run's start and best
    warm = [(0, 100.8), (5, 100.1)]
    assert study.within_gap(warm, 200.0, 100.0) == 0
    assert study.within_gap(warm, 200.0, 100.0, frac=0.005) == 5


def test_asset_classes_partition_the_plan():
    nets, _ = synth.medium(S=1, T=24)
    g = study.asset_classes(nets[0])
    allix = np.concatenate(list(g.values()))
    assert np.array_equal(np.sort(allix), np.arange(nets[0]["K"]))
    assert g["gas"].size + g["solar"].size + g["wind"].size == nets[0]["gen_bus"].size


def test_autotune_accuracy_guard():
    from paper_2410_13055_gb300 import autotune
    assert autotune.accept(100.1, 100.0, 0.03, 0.03)              # objective 1e-3 off, same gradient error
    assert not autotune.accept(100.3, 100.0, 0.03, 0.03)          # objective 3e-3 off
    assert autotune.accept(-100.1, -100.0, 0.0375, 0.03)          # gradient error at the 1.25x slack
    assert not autotune.accept(100.0, 100.0, 0.04, 0.03)          # gradient error beyond the slack
    assert autotune.accept(100.0, 100.0, 0.01, 0.03, g_slack=1.0)  # more accurate than the defaults
