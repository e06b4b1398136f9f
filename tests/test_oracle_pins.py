"""Pins of the CPU oracle to facts outside itself (no GPU).

Each pin_* function raises AssertionError when the oracle library it is
given disagrees with a closed form, a textbook routine, brute force, a
hand-worked example or an invariant.  The tests run them on the oracle; the
mutation test (test_oracle_mutants.py) plants plausible mistakes in a copy of
the oracle source and checks that some pin fails for each.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import norm

from oracle import oracle
from paper_2101_05012_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
E0 = -0.91893853320467274178          # ln(1/sqrt(2 pi))


# ----------------------------------------------------------------------------
# constants: closed forms of Alg. adaptivebandedcpucompute's constants

def pin_constants(lib):
    # ln(a - 1e-10) = ln(a) - 1e-10/a to 1e-19, so every value below is a
    # closed form: lp_stay = ln(1 - 1/(epk+1)), lp_step = ln(1/(epk+1) - 1e-10).
    cases = {
        (3, 2): (-0.5108256237659907, -0.9162907321241551),   # epk 1.5: ln(3/5), ln(2/5) - 2.5e-10
        (2, 1): (-0.4054651081081644, -1.0986122889681098),   # epk 2:   ln(2/3), ln(1/3) - 3e-10
        (5, 2): (-0.3364722366212129, -1.2527629688453680),   # epk 2.5: ln(5/7), ln(2/7) - 3.5e-10
        (1, 1): (-0.6931471805599453, -0.6931471807599453),   # epk 1:   ln(1/2), ln(1/2) - 2e-10
    }
    for (ne, nk), (stay, step) in cases.items():
        skip_, stay_, step_, trim_ = oracle.constants(ne, nk, lib=lib)
        assert abs(skip_ - (-23.025850929940457)) < 1e-13, skip_     # ln(1e-10)
        assert abs(trim_ - (-4.605170185988091)) < 1e-13, trim_       # ln(1/100)
        assert abs(stay_ - stay) < 1e-13, (ne, nk, stay_)
        assert abs(step_ - step) < 1e-13, (ne, nk, step_)


def test_constants(olib):
    pin_constants(olib)


# ----------------------------------------------------------------------------
# emission: one event on one k-mer aligns by a single D step from the origin,
# so the score is lp_step + log N(x; scale*mu + shift, var*sigma).

def _one_cell(lib, x, mu, sd, sc, precision):
    r = oracle.abea([mu, 0, 0, 0], [sd, 1, 1, 1], 1, "A", [x], sc, 4, precision, lib=lib)
    assert r["status"] == oracle.ST_OK
    assert r["pairs"].tolist() == [[0, 0]]
    return r["score"]


def pin_emission(lib, precision="f64"):
    lp_step_epk1 = -0.6931471807599453      # ln(1/2 - 1e-10) = ln(1/2) - 2e-10 to 1e-19
    tol = 1e-9 if precision == "f64" else 3e-6
    # x on the mean, sigma' = 1: ln(1/sqrt(2 pi))
    s = _one_cell(lib, 100.0, 100.0, 1.0, (1, 0, 1), precision)
    assert abs(s - (lp_step_epk1 + E0)) < tol, s
    # sigma' = 2: ln 2 less; and sigma = 1, var = 2 gives the same (sigma' = var*sigma)
    s = _one_cell(lib, 100.0, 100.0, 2.0, (1, 0, 1), precision)
    assert abs(s - (lp_step_epk1 + E0 - 0.6931471805599453)) < tol, s
    s = _one_cell(lib, 100.0, 100.0, 1.0, (1, 0, 2), precision)
    assert abs(s - (lp_step_epk1 + E0 - 0.6931471805599453)) < tol, s
    # one sigma' away: a further -1/2; the mean is scale*mean + shift
    s = _one_cell(lib, 103.0, 50.0, 1.5, (2, 0, 2), precision)
    assert abs(s - (lp_step_epk1 + E0 - 1.0986122886681098 - 0.5)) < tol, s
    # random points against the textbook density (scipy), with scalings
    rng = np.random.default_rng(7)
    for _ in range(200):
        mu = float(np.float32(rng.uniform(60, 130)))
        sd = float(np.float32(rng.uniform(1, 3)))
        scale = float(np.float32(rng.uniform(0.9, 1.1)))
        shift = float(np.float32(rng.uniform(-5, 5)))
        var = float(np.float32(rng.uniform(1, 1.5)))
        # |z| <= 4 keeps the D step (lp_step + emission) above the trim-then-skip
        # entry (lp_trim + lp_skip = -27.6), so the score is the emission's
        x = float(np.float32(scale * mu + shift + rng.uniform(-4, 4) * sd * var))
        want = lp_step_epk1 + norm.logpdf(x, loc=scale * mu + shift, scale=var * sd)
        got = _one_cell(lib, x, mu, sd, (scale, shift, var), precision)
        assert abs(got - want) <= tol * max(1.0, abs(want)), (got, want, x, mu, sd, scale, shift, var)


def test_emission_f64(olib):
    pin_emission(olib, "f64")


def test_emission_f32(olib):
    pin_emission(olib, "f32")


# ----------------------------------------------------------------------------
# brute force: every monotone path of the augmented grid, tiny inputs

def _brute_force(model_mean, model_stdv, k, seq, events, sc, lib):
    """Best score over every monotone path, the best path, and whether that
    path is the unique optimum (the runner-up is more than 1e-6 behind)."""
    n_e = len(events)
    ranks = oracle.kmer_ranks(seq, k, lib=lib)
    n_k = len(ranks)
    lp_skip, lp_stay, lp_step, lp_trim = oracle.constants(n_e, n_k, lib=lib)
    scale, shift, var = sc
    E = np.array([[norm.logpdf(float(events[e]), loc=scale * float(model_mean[r]) + shift,
                               scale=var * float(model_stdv[r])) for r in ranks] for e in range(n_e)])
    found = {}

    def walk(e, kk, score, path):
        path = path + ((e, kk),)
        if kk == n_k - 1:
            cand = score + (n_e - 1 - e) * lp_trim
            found[path] = max(found.get(path, -math.inf), cand)
        if e + 1 < n_e and kk + 1 < n_k:
            walk(e + 1, kk + 1, score + lp_step + E[e + 1, kk + 1], path)
        if e + 1 < n_e:
            walk(e + 1, kk, score + lp_stay + E[e + 1, kk], path)
        if kk + 1 < n_k:
            walk(e, kk + 1, score + lp_skip, path)

    # enter the matrix from the origin (-1,-1) or from a trim cell (e,-1)
    walk(0, 0, lp_step + E[0, 0], ())
    for e in range(n_e):
        t = (e + 1) * lp_trim
        if e + 1 < n_e:
            walk(e + 1, 0, t + lp_step + E[e + 1, 0], ())
        walk(e, 0, t + lp_skip, ())
    ranked = sorted(found.items(), key=lambda kv: -kv[1])
    best_path, best = ranked[0]
    unique = len(ranked) == 1 or ranked[1][1] < best - 1e-6
    return best, [list(p) for p in best_path], unique


def _tiny_cases(n_cases, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n_cases):
        k = int(rng.integers(1, 3))
        n_model = 4 ** k
        mm = rng.uniform(60, 130, n_model).astype(np.float32)
        ms = rng.uniform(1, 8, n_model).astype(np.float32)
        n_k = int(rng.integers(1, 5))
        n_e = int(rng.integers(1, 5))
        seq = "".join(rng.choice(list("ACGT"), n_k + k - 1))
        ev = rng.uniform(60, 130, n_e).astype(np.float32)
        sc = (float(np.float32(rng.uniform(0.9, 1.1))), float(np.float32(rng.uniform(-5, 5))),
              float(np.float32(rng.uniform(1, 1.5))))
        yield mm, ms, k, seq, ev, sc


def pin_brute_force(lib, n_cases=60, seed=11):
    n_unique = 0
    for mm, ms, k, seq, ev, sc in _tiny_cases(n_cases, seed):
        want, path, unique = _brute_force(mm, ms, k, seq, ev, sc, lib)
        n_unique += unique
        full = oracle.full_dp(mm, ms, k, seq, ev, sc, "f64", lib=lib)
        n = max(len(ev), len(seq) - k + 1)
        band = oracle.abea(mm, ms, k, seq, ev, sc, 2 * n + 8, "f64", lib=lib)
        for r in (full, band):
            assert r["status"] == oracle.ST_OK
            assert abs(r["score"] - want) < 1e-9 * max(1, abs(want)), (r["score"], want, seq, ev)
            got = r["pairs"].tolist()
            if unique:
                assert got == path, (got, path)
            else:   # several optimal paths: the reported one must be one of them
                assert abs(rescore(got, mm, ms, k, seq, ev, sc, lib) - want) < 1e-9 * max(1, abs(want))
    assert n_unique >= n_cases // 2


def test_brute_force(olib):
    pin_brute_force(olib)


# ----------------------------------------------------------------------------
# wide band reduces to the full DP; every augmented cell lies in its band

def pin_wide_band_is_full_dp(lib, n_reads=6):
    b = synth.make_batch(synth.Workload("wide", n_reads, 3, 0, 21, ("fixed", 40)))
    for i in range(b.n):
        ev, sq, sc = b.read(i)
        n_e, n_k = len(ev), len(sq) - b.k + 1
        W = 2 * max(n_e, n_k) + 8
        r = oracle.abea(b.model_mean, b.model_stdv, b.k, sq, ev, sc, W, "f64", with_bands=True, lib=lib)
        ll = r["ll"]
        # every cell (e,k) of [-1,n_e) x [-1,n_k) sits at a valid offset of band e+k+2
        for e in range(-1, n_e):
            for kk in range(-1, n_k):
                bb = e + kk + 2
                j = ll[bb, 0] - e
                assert 0 <= j < W and ll[bb, 1] + j == kk, (e, kk, bb, j)
        f = oracle.full_dp(b.model_mean, b.model_stdv, b.k, sq, ev, sc, "f64", lib=lib)
        assert r["score"] == f["score"], (r["score"], f["score"])
        assert np.array_equal(r["pairs"], f["pairs"])
        assert r["cells"] == n_e * n_k


def test_wide_band_is_full_dp(olib):
    pin_wide_band_is_full_dp(olib)


# ----------------------------------------------------------------------------
# hand-worked examples (tests/golden/hand_examples.json)

def pin_hand_examples(lib, precision="f64"):
    g = json.load(open(GOLDEN))
    for ex in g["examples"]:
        ev = np.array(ex["events"], np.float32)
        n_e, n_k = len(ev), len(ex["seq"])
        epk = n_e / n_k
        lp_stay = math.log(1 - 1 / (epk + 1))
        vals = {"E0": E0, "lp_trim": math.log(0.01), "lp_skip": math.log(1e-10), "lp_stay": lp_stay,
                "lp_step": math.log(1 - 1e-10 - math.exp(lp_stay))}
        want = sum(vals[t] for t in ex["terms"])
        for W in (4, 8, 100):
            r = oracle.abea(g["model_levels"], g["model_stdv"], 1, ex["seq"], ev, (1, 0, 1), W, precision, lib=lib)
            assert r["status"] == oracle.ST_OK, ex["name"]
            assert r["pairs"].tolist() == ex["pairs"], (ex["name"], W, r["pairs"].tolist())
            assert abs(r["score"] - want) < (1e-9 if precision == "f64" else 1e-5), (ex["name"], r["score"], want)


def test_hand_examples_f64(olib):
    pin_hand_examples(olib, "f64")


def test_hand_examples_f32(olib):
    pin_hand_examples(olib, "f32")


# ----------------------------------------------------------------------------
# band positions while both band ends are -inf: the alternation rule of the
# author comment in Alg. adaptivebandedcpu (k-mer move on odd bands), worked
# by hand for W = 8 and W = 9 (tests/golden/band_positions.json)

BANDS_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "band_positions.json")


def pin_band_positions(lib):
    g = json.load(open(BANDS_GOLDEN))
    rd = g["read"]
    rng = np.random.default_rng(rd["seed"])
    k = rd["k"]
    mm = rng.uniform(60, 130, 4 ** k).astype(np.float32)
    ms = rng.uniform(1, 3, 4 ** k).astype(np.float32)
    seq = "".join(rng.choice(list("ACGT"), rd["n_bases"]))
    ev = rng.uniform(60, 130, rd["n_events"]).astype(np.float32)
    for case in g["cases"]:
        for precision in ("f64", "f32"):
            r = oracle.abea(mm, ms, k, seq, ev, (1.0, 0.0, 1.0), case["W"], precision, with_bands=True, lib=lib)
            assert r["status"] == oracle.ST_OK
            want = case["ll"]
            assert r["ll"][:len(want)].tolist() == want, (case["W"], precision, r["ll"][:len(want)].tolist())


def test_band_positions(olib):
    pin_band_positions(olib)


# ----------------------------------------------------------------------------
# invariants on realistic reads; re-scoring the path from its pairs

def rescore(pairs, model_mean, model_stdv, k, seq, events, sc, lib):
    """Score of a path recomputed from its pairs in FP64 (scipy emissions)."""
    n_e = len(events)
    ranks = oracle.kmer_ranks(seq, k, lib=lib)
    lp_skip, lp_stay, lp_step, lp_trim = oracle.constants(n_e, len(ranks), lib=lib)
    scale, shift, var = sc

    def em(e, kk):
        r = ranks[kk]
        return norm.logpdf(float(events[e]), loc=scale * float(model_mean[r]) + shift,
                           scale=var * float(model_stdv[r]))
    e0, k0 = pairs[0]
    # entry: from (e0-1,-1) by a D step, or from the trim cell (e0,-1) by an L step
    s = max(e0 * lp_trim + lp_step + em(e0, 0), (e0 + 1) * lp_trim + lp_skip)
    for (pe, pk), (e, kk) in zip(pairs[:-1], pairs[1:]):
        if (e - pe, kk - pk) == (1, 1):
            s += lp_step + em(e, kk)
        elif (e - pe, kk - pk) == (1, 0):
            s += lp_stay + em(e, kk)
        else:
            s += lp_skip
    return s + (n_e - 1 - pairs[-1][0]) * lp_trim


def pin_invariants(lib, n_reads=6):
    b = synth.make_batch("plain_64x1kb", n_reads=n_reads)
    for i in range(b.n):
        ev, sq, sc = b.read(i)
        n_e, n_k = len(ev), len(sq) - b.k + 1
        r = oracle.abea(b.model_mean, b.model_stdv, b.k, sq, ev, sc, b.W, "f64", with_bands=True, lib=lib)
        assert r["status"] == oracle.ST_OK
        ll, W = r["ll"], b.W
        nb = n_e + n_k + 1
        assert ll.shape[0] == nb
        assert tuple(ll[0]) == (W // 2 - 1, -1 - W // 2) and tuple(ll[1]) == (W // 2, -1 - W // 2)
        d = np.diff(ll, axis=0)
        assert np.all(d.sum(axis=1) == 1) and np.all((d == 0) | (d == 1))     # one index advances per band
        assert np.all(ll.sum(axis=1) == np.arange(nb) - 2)                   # e + k = b - 2
        for bb in range(nb):                                                 # band meets the augmented matrix
            j = np.arange(W)
            e, kk = ll[bb, 0] - j, ll[bb, 1] + j
            assert np.any((e >= -1) & (e < n_e) & (kk >= -1) & (kk < n_k)), bb
        p = r["pairs"]
        assert p[0, 1] == 0 and p[-1, 1] == n_k - 1
        steps = np.diff(p, axis=0)
        assert all(tuple(s) in ((1, 1), (1, 0), (0, 1)) for s in steps)
        assert np.all(np.diff(p.sum(axis=1)) > 0)
        assert p[-1, 0] == r["e_end"]
        s = rescore(p.tolist(), b.model_mean, b.model_stdv, b.k, sq, ev, sc, lib)
        assert abs(s - r["score"]) < 1e-9 * abs(s), (s, r["score"])
        # cells: in-matrix offsets of bands 2.. (from the band positions)
        cells = 0
        for bb in range(2, nb):
            j = np.arange(W)
            e, kk = ll[bb, 0] - j, ll[bb, 1] + j
            cells += int(np.sum((e >= 0) & (e < n_e) & (kk >= 0) & (kk < n_k)))
        assert cells == r["cells"]


def test_invariants(olib):
    pin_invariants(olib)


# ----------------------------------------------------------------------------
# the vectorised FP64 path scorer (oracle/rescore.py, used by the FP64
# accuracy checks) against the oracle's own FP64 scores and the hand examples

def test_path_scores_reproduce_fp64_scores(olib):
    from oracle import rescore
    b = synth.make_batch("plain_64x1kb", n_reads=12)
    o = oracle.abea_batch(b, "f64", n_threads=4, lib=olib)
    s = rescore.path_scores(b, o["pairs"], o["pair_off"], o["n_pairs"], o["status"] == oracle.ST_OK)
    assert np.all(o["status"] == oracle.ST_OK)
    assert np.max(np.abs(s - o["score"]) / np.abs(o["score"])) < 1e-11
    # a path with one pair moved off the optimum scores lower
    p = o["pairs"].copy()
    i = int(o["pair_off"][0]) + 5
    p[i:i + 1, 1] = p[i + 1, 1] if p[i + 1, 1] != p[i, 1] else p[i, 1]
    s2 = rescore.path_scores(b, p, o["pair_off"], o["n_pairs"], o["status"] == oracle.ST_OK)
    assert s2[0] <= s[0]


def test_path_scores_hand_examples():
    from oracle import rescore
    g = json.load(open(GOLDEN))
    for ex in g["examples"]:
        ev = np.array(ex["events"], np.float32)
        n_e, n_k = len(ev), len(ex["seq"])
        lp_stay = math.log(1 - 1 / (n_e / n_k + 1))
        vals = {"E0": E0, "lp_trim": math.log(0.01), "lp_skip": math.log(1e-10), "lp_stay": lp_stay,
                "lp_step": math.log(1 - 1e-10 - math.exp(lp_stay))}
        want = sum(vals[t] for t in ex["terms"])
        b = synth.custom_batch([ev], [ex["seq"].encode()], [(1.0, 0.0, 1.0)], np.asarray(g["model_levels"], np.float32),
                               np.asarray(g["model_stdv"], np.float32), 1, 4)
        pairs = np.asarray(ex["pairs"], np.int32)
        s = rescore.path_scores(b, pairs, np.array([0, len(pairs)]), np.array([len(pairs)]), np.array([True]))
        assert abs(s[0] - want) < 1e-9 * abs(want), (ex["name"], s[0], want)


# ----------------------------------------------------------------------------
# FP32 oracle against FP64: score within 1e-4 relative; same path when no
# near-tie (< 1e-3) decision was taken in FP64.

def test_fp32_vs_fp64(olib):
    b = synth.make_batch("plain_64x1kb", n_reads=16)
    r64 = oracle.abea_batch(b, "f64", n_threads=4)
    r32 = oracle.abea_batch(b, "f32", n_threads=4)
    assert np.all(r64["status"] == 0) and np.all(r32["status"] == 0)
    rel = np.abs(r32["score"] - r64["score"]) / np.abs(r64["score"])
    assert rel.max() <= 1e-4, rel.max()
    for i in range(b.n):
        if r64["min_margin"][i] >= 1e-3:
            a = r64["pairs"][r64["pair_off"][i]:r64["pair_off"][i] + r64["n_pairs"][i]]
            c = r32["pairs"][r32["pair_off"][i]:r32["pair_off"][i] + r32["n_pairs"][i]]
            assert np.array_equal(a, c), i


# ----------------------------------------------------------------------------
# FP32 on long reads (where the exact renormalisation of the FP32 form acts)
# against FP64: same path unless near-tie, score within 2e-5 relative.

def pin_fp32_long_read(lib):
    w = synth.Workload("long", 2, 6, 100, 31, ("fixed", 20_000))
    b = synth.make_batch(w)
    for i in range(b.n):
        ev, sq, sc = b.read(i)
        r64 = oracle.abea(b.model_mean, b.model_stdv, b.k, sq, ev, sc, b.W, "f64", lib=lib)
        r32 = oracle.abea(b.model_mean, b.model_stdv, b.k, sq, ev, sc, b.W, "f32", lib=lib)
        assert r64["status"] == r32["status"] == oracle.ST_OK
        assert abs(r32["score"] - r64["score"]) <= 2e-5 * abs(r64["score"]), (r32["score"], r64["score"])
        if r64["min_margin"] >= 1e-3:
            assert np.array_equal(r32["pairs"], r64["pairs"])


def test_fp32_long_read(olib):
    pin_fp32_long_read(olib)


# ----------------------------------------------------------------------------
# degenerate inputs

def test_degenerate(olib):
    mm = [60.0, 80.0, 100.0, 120.0]
    ms = [1.0] * 4
    # one event, one k-mer
    r = oracle.abea(mm, ms, 1, "G", [100.0], (1, 0, 1), 2, "f64", lib=olib)
    assert r["status"] == 0 and r["pairs"].tolist() == [[0, 0]]
    # W = 2 still aligns a short read end to end
    r = oracle.abea(mm, ms, 1, "ACGT", [60, 80, 100, 120], (1, 0, 1), 2, "f64", lib=olib)
    assert r["status"] == 0 and r["pairs"].tolist() == [[0, 0], [1, 1], [2, 2], [3, 3]]
    # invalid inputs
    for args in [("ACNT", [60.0], (1, 0, 1), 10),            # non-ACGT base
                 ("ACGT", [], (1, 0, 1), 10),                # no events
                 ("ACGT", [float("nan")], (1, 0, 1), 10),    # NaN event
                 ("ACGT", [60.0], (1, 0, 0), 10),            # var = 0
                 ("ACGT", [60.0], (1, 0, 1), 1)]:            # W < 2
        r = oracle.abea(mm, ms, 1, args[0], args[1], args[2], args[3], "f64", lib=olib)
        assert r["status"] == oracle.ST_BAD_INPUT, args
    # sequence shorter than k
    r = oracle.abea(np.zeros(16, np.float32) + 80, np.ones(16, np.float32), 2, "A", [60.0], (1, 0, 1), 4, "f64", lib=olib)
    assert r["status"] == oracle.ST_BAD_INPUT
