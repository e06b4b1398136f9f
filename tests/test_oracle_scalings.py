"""Pins of the scaling-estimate oracle (method of moments, population
moments): hand-worked values, exact recovery of an affine map, invariances,
degenerate and rejected reads, and planted mistakes that must fail a pin."""
import numpy as np
import pytest

from oracle import scalings_oracle as so

K1_LEVELS = np.array([60.0, 80.0, 100.0, 120.0])          # k = 1: A C G T


def test_hand_example_one_event_per_kmer():
    # levels 60, 80, 100, 120: mean 90, population variance 500; events = 2 * level + 10
    scale, shift, st = so.estimate(K1_LEVELS, 1, "ACGT", [130.0, 170.0, 210.0, 250.0])
    assert st == so.SC_OK
    assert scale == pytest.approx(2.0, abs=1e-14) and shift == pytest.approx(10.0, abs=1e-12)


def test_hand_example_population_moments():
    # six events over four k-mers: event mean 190, population variance 15200 / 6;
    # levels: mean 90, population variance 500 -> scale = sqrt(15200 / 3000)
    ev = [130.0, 130.0, 170.0, 210.0, 250.0, 250.0]
    scale, shift, st = so.estimate(K1_LEVELS, 1, "ACGT", ev)
    want = np.sqrt(15200.0 / 3000.0)                      # 2.25092573...
    assert st == so.SC_OK
    assert scale == pytest.approx(want, rel=1e-14)
    assert shift == pytest.approx(190.0 - want * 90.0, rel=1e-13)


def test_exact_affine_recovery_random():
    rng = np.random.default_rng(11)
    k = 6
    levels = rng.uniform(60, 130, 4 ** k)
    for _ in range(20):
        seq = "".join(rng.choice(list("ACGT"), rng.integers(8, 400)))
        a, b = rng.uniform(0.8, 1.3), rng.uniform(-8, 8)
        ranks = np.array([int("".join("ACGT".index(c).__str__() for c in seq[i:i + k]), 4)
                          for i in range(len(seq) - k + 1)])
        ev = a * levels[ranks] + b
        scale, shift, st = so.estimate(levels, k, seq, ev)
        assert st == so.SC_OK
        assert scale == pytest.approx(a, rel=1e-11) and shift == pytest.approx(b, abs=1e-8)


def test_affine_equivariance_and_permutation_invariance():
    rng = np.random.default_rng(12)
    levels = rng.uniform(60, 130, 4 ** 3)
    seq = "".join(rng.choice(list("ACGT"), 300))
    ev = rng.normal(95, 12, 500)
    s0, h0, _ = so.estimate(levels, 3, seq, ev)
    alpha, beta = 1.7, -4.25
    s1, h1, _ = so.estimate(levels, 3, seq, alpha * ev + beta)
    assert s1 == pytest.approx(alpha * s0, rel=1e-12) and h1 == pytest.approx(alpha * h0 + beta, rel=1e-12)
    s2, h2, _ = so.estimate(levels, 3, seq, rng.permutation(ev))
    assert s2 == pytest.approx(s0, rel=1e-12) and h2 == pytest.approx(h0, rel=1e-12)


def test_degenerate_and_rejected_reads():
    # one k-mer rank only: the levels have no variance
    s, h, st = so.estimate(K1_LEVELS, 1, "AAAAAA", [70.0, 75.0, 80.0])
    assert st == so.SC_DEGENERATE and s == 1.0 and h == pytest.approx(75.0 - 60.0)
    # a single event
    s, h, st = so.estimate(K1_LEVELS, 1, "ACGT", [100.0])
    assert st == so.SC_DEGENERATE and s == 1.0 and h == pytest.approx(10.0)
    # constant events
    s, h, st = so.estimate(K1_LEVELS, 1, "ACGT", [95.0, 95.0])
    assert st == so.SC_DEGENERATE and h == pytest.approx(5.0)
    for seq, ev in (("ACNT", [1.0, 2.0]), ("ACGT", []), ("", [1.0, 2.0]), ("ACGT", [1.0, np.nan])):
        assert so.estimate(K1_LEVELS, 1, seq, ev)[2] == so.SC_BAD_INPUT
    assert so.estimate(K1_LEVELS[:4], 1, "ACGT", [1.0, np.inf])[2] == so.SC_BAD_INPUT


# Planted mistakes: each must fail at least one pin above.
def _sample_variance(model_mean, k, seq, events):
    ev = np.asarray(events, float)
    mu = np.asarray(model_mean, float)[[("ACGT".index(c)) for c in seq]] if k == 1 else None
    scale = np.sqrt(ev.var(ddof=1) / mu.var(ddof=1))
    return scale, ev.mean() - scale * mu.mean(), so.SC_OK


def _inverted_scale(model_mean, k, seq, events):
    s, h, st = so.estimate(model_mean, k, seq, events)
    return 1.0 / s, h, st


def _shift_without_scale(model_mean, k, seq, events):
    s, h, st = so.estimate(model_mean, k, seq, events)
    ev = np.asarray(events, float)
    mu = np.asarray(model_mean, float)[[("ACGT".index(c)) for c in seq]]
    return s, ev.mean() - mu.mean(), st


@pytest.mark.parametrize("mutant", [_sample_variance, _inverted_scale, _shift_without_scale])
def test_planted_mistakes_fail_a_pin(mutant):
    failures = 0
    for ev, want_scale, want_shift in (([130.0, 170.0, 210.0, 250.0], 2.0, 10.0),
                                       ([130.0, 130.0, 170.0, 210.0, 250.0, 250.0], np.sqrt(15200 / 3000),
                                        190.0 - np.sqrt(15200 / 3000) * 90.0)):
        s, h, _ = mutant(K1_LEVELS, 1, "ACGT", ev)
        if abs(s - want_scale) > 1e-9 or abs(h - want_shift) > 1e-6:
            failures += 1
    assert failures > 0
