"""Pins of the event-detection oracle: a hand-worked t2 example, exact
segmentation of noiseless steps, the tie rule, shift invariance, event
statistics against FP64 definitions, and planted mistakes that must fail."""
import numpy as np
import pytest

from oracle import event_oracle as eo

CAL = (0.0, 1.0)


def test_hand_example_t2_and_events():
    # w = 2, x = 10 10 10 20 20 20:
    #   i=2: S_L=20 S_R=30 Q_L=200 Q_R=500 -> N=2*10^2=200, D=2*700-400-900=100 -> 2
    #   i=3: S_L=20 S_R=40 Q_L=200 Q_R=800 -> N=800, D=2000-400-1600=0 -> inf
    #   i=4: S_L=30 S_R=40 Q_L=500 Q_R=800 -> N=200, D=2600-900-1600=100 -> 2
    x = np.array([10, 10, 10, 20, 20, 20], np.int16)
    t2 = eo.t2_values(x, 2)
    assert list(t2) == [0.0, 0.0, 2.0, np.inf, 2.0, 0.0]
    m, s, a, L = eo.detect(x, 2, 1.0, CAL)
    assert list(a) == [0, 3] and list(L) == [3, 3] and list(m) == [10.0, 20.0] and list(s) == [0.0, 0.0]


def test_noiseless_steps_are_found_exactly():
    rng = np.random.default_rng(5)
    for w in (2, 3, 5):
        lens = rng.integers(2 * w, 6 * w, 40)
        levels = rng.integers(200, 900, 40)
        levels[1:] += (levels[1:] == levels[:-1])            # no two equal neighbours
        x = np.repeat(levels, lens).astype(np.int16)
        m, s, a, L = eo.detect(x, w, 1e-3, (2.5, 0.5))
        assert np.array_equal(a, np.concatenate([[0], np.cumsum(lens)[:-1]]))
        assert np.array_equal(L, lens)
        assert np.array_equal(m, ((levels + np.float32(2.5)) * np.float32(0.5)).astype(np.float32))
        assert np.all(s == 0)


def test_tie_rule_and_threshold():
    t2 = np.array([0, 5, 5, 0, 0, 0, 0, 3, 0, 4, 0], np.float32)
    # w = 3: 1 and 2 tie -> the earlier; 7 and 9 are 2 apart, 9 is larger -> 9 only
    assert list(eo.boundaries(t2, 3, 1.0)) == [1, 9]
    assert list(eo.boundaries(t2, 3, 4.0)) == [1, 9]              # t2 >= tau2 keeps 4
    assert list(eo.boundaries(t2, 3, 4.5)) == [1]
    assert list(eo.boundaries(t2, 2, 1.0)) == [1, 7, 9]           # 7 and 9 are 2 apart: both stand


def test_shift_invariance_and_statistics():
    rng = np.random.default_rng(6)
    x = (rng.normal(500, 20, 3000) + np.repeat(rng.integers(0, 300, 300), 10)).astype(np.int16)
    b0 = eo.boundaries(eo.t2_values(x, 3), 3, 2.0)
    b1 = eo.boundaries(eo.t2_values(x + np.int16(1000), 3), 3, 2.0)
    assert np.array_equal(b0, b1)
    m, s, a, L = eo.detect(x, 3, 2.0, (-3.0, 0.25))
    for e in range(0, len(a), 37):
        seg = x[a[e]:a[e] + L[e]].astype(np.float64)
        assert m[e] == pytest.approx((seg.mean() - 3.0) * 0.25, rel=2e-6)
        assert s[e] == pytest.approx(seg.std() * 0.25, rel=2e-3, abs=2e-3)
    assert L.sum() == len(x) and a[0] == 0 and np.all(np.diff(a) == L[:-1])


def test_short_and_empty_signals():
    assert len(eo.detect(np.zeros(0, np.int16), 3, 2.0, CAL)[0]) == 0
    m, s, a, L = eo.detect(np.array([5, 9, 7], np.int16), 3, 2.0, CAL)     # shorter than two windows
    assert list(a) == [0] and list(L) == [3] and m[0] == np.float32(21) / np.float32(3)


# Planted mistakes: each must fail one of the checks below (the pins above in small form).
def _ties_to_latest(t2, w, tau2):
    n = len(t2)
    return np.array([i for i in range(1, n) if t2[i] >= tau2
                     and not any(t2[j] > t2[i] for j in range(max(0, i - w + 1), i))
                     and not any(t2[j] >= t2[i] for j in range(i + 1, min(n, i + w)))], np.int64)


def _strict_threshold(t2, w, tau2):
    return np.array([i for i in eo.boundaries(t2, w, tau2) if t2[i] > tau2], np.int64)


def _one_sided_window(t2, w, tau2):
    n = len(t2)
    return np.array([i for i in range(1, n) if t2[i] >= tau2
                     and not any(t2[j] >= t2[i] for j in range(max(0, i - w + 1), i))], np.int64)


@pytest.mark.parametrize("mutant", [_ties_to_latest, _strict_threshold, _one_sided_window])
def test_planted_mistakes_fail(mutant):
    t2 = np.array([0, 5, 5, 0, 0, 0, 0, 3, 0, 4, 0], np.float32)
    cases = [((t2, 3, 1.0), [1, 9]), ((t2, 3, 4.0), [1, 9]), ((t2, 2, 1.0), [1, 7, 9])]
    assert any(list(mutant(*args)) != want for args, want in cases)
