"""FP64 score of given alignment paths, from the recurrence's definition.

TEST INFRASTRUCTURE ONLY: used by tests/ and by the CPU-baseline leg of
bench.py, never by the product path.

A path (pairs of event and k-mer index, ascending) scores, in the thesis's
formulas (Ch.5, Alg. adaptivebandedcpucompute and ...computelog, with the
read-model scaling of Sec. ABEA and the trim states):
  * its first pair (e0, 0) is entered from the trim column, either from
    (e0-1, -1) by a diagonal step (that trim cell scores e0*ln(1/100); the
    origin for e0 = 0) or from (e0, -1) by a skip ((e0+1)*ln(1/100) + lp_skip),
    whichever scores more (the recurrence keeps the better);
  * each later pair adds lp_step + E (event and k-mer both advance), lp_stay + E
    (event only) or lp_skip (k-mer only), where E = log N(x_e; mu', sigma'),
    mu' = scale*mean + shift, sigma' = var*stdv;
  * the events after the last pair are trimmed at ln(1/100) each.
Every read's path is scored at once with numpy (no banding: a path is scored
as given, whether or not its cells lie in a band).
"""
from __future__ import annotations

import numpy as np

LOG_INV_SQRT_2PI = -0.91893853320467274178


def transition_constants(n_events, n_kmers):
    """(lp_skip, lp_stay, lp_step, lp_trim) per read, FP64."""
    epk = np.asarray(n_events, np.float64) / np.asarray(n_kmers, np.float64)
    lp_skip = np.log(1e-10)
    lp_stay = np.log(1.0 - 1.0 / (epk + 1.0))
    lp_step = np.log(1.0 - np.exp(lp_skip) - np.exp(lp_stay))
    return lp_skip, lp_stay, lp_step, np.log(1.0 / 100.0)


def path_scores(batch, pairs, pair_off, n_pairs, valid):
    """FP64 score of read i's path pairs[pair_off[i] : pair_off[i] + n_pairs[i]] for every read with
    valid[i] (others: -inf).  pairs is int32[P, 2] (event, k-mer)."""
    n = batch.n
    n_e = batch.n_events().astype(np.int64)
    n_k = batch.n_kmers().astype(np.int64)
    lp_skip, lp_stay, lp_step, lp_trim = transition_constants(n_e, np.maximum(n_k, 1))
    cnt = np.where(np.asarray(valid), np.asarray(n_pairs), 0).astype(np.int64)
    total = int(cnt.sum())
    out = np.full(n, -np.inf)
    if total == 0:
        return out
    rid = np.repeat(np.arange(n), cnt)
    first_of = np.cumsum(cnt) - cnt
    local = np.arange(total) - np.repeat(first_of, cnt)
    p = np.asarray(pairs).reshape(-1, 2)[np.repeat(np.asarray(pair_off[:n], np.int64), cnt) + local]
    e = p[:, 0].astype(np.int64)
    k = p[:, 1].astype(np.int64)
    # k-mer ranks: lexicographic over ACGT, first base most significant
    code = np.full(256, 0, np.int64)
    for c, v in zip(b"ACGT", range(4)):
        code[c] = v
    bases = code[batch.seq]
    pos = np.asarray(batch.seq_off, np.int64)[rid] + k
    rank = np.zeros(total, np.int64)
    for t in range(batch.k):
        rank = rank * 4 + bases[pos + t]
    x = batch.events[np.asarray(batch.ev_off, np.int64)[rid] + e].astype(np.float64)
    sc = np.asarray(batch.scalings, np.float64)
    mu = batch.model_mean[rank].astype(np.float64) * sc[rid, 0] + sc[rid, 1]
    sd = batch.model_stdv[rank].astype(np.float64) * sc[rid, 2]
    z = (x - mu) / sd
    em = LOG_INV_SQRT_2PI - np.log(sd) - 0.5 * z * z
    first = local == 0
    prev = np.maximum(np.arange(total) - 1, 0)
    de = e - e[prev]
    dk = k - k[prev]
    step = np.where((de == 1) & (dk == 1), lp_step[rid] + em,
                    np.where((de == 1) & (dk == 0), lp_stay[rid] + em, lp_skip))
    entry = np.maximum(e * lp_trim + lp_step[rid] + em, (e + 1) * lp_trim + lp_skip)
    s = np.bincount(rid, weights=np.where(first, entry, step), minlength=n)
    e_last = e[np.maximum(np.cumsum(cnt) - 1, 0)]
    s = s + (n_e - 1 - e_last) * lp_trim
    out[cnt > 0] = s[cnt > 0]
    return out


def accuracy_against_fp64(batch, res, pairs, pair_off, o64, near_tie=1e-3):
    """Accuracy of FP32 results (res: score, status, n_pairs; pairs at pair_off) against the FP64
    oracle's results o64 on the same reads: the near-tie fraction (reads whose FP64 run took a decision
    by less than `near_tie`), path mismatches among the other reads, the largest relative score
    error, and the largest gap between the FP64 optimum and the FP64 score of the FP32 path."""
    ok = (np.asarray(res["status"]) == 0) & (np.asarray(o64["status"]) == 0)
    tie = np.asarray(o64["min_margin"]) < near_tie
    exact = np.asarray(o64["min_margin"]) == 0.0
    mism = 0
    for i in np.nonzero(ok & ~tie)[0]:
        a = pairs[pair_off[i]:pair_off[i] + res["n_pairs"][i]]
        b = o64["pairs"][o64["pair_off"][i]:o64["pair_off"][i] + o64["n_pairs"][i]]
        if not np.array_equal(a, b):
            mism += 1
    rel = np.abs(np.asarray(res["score"], np.float64)[ok] - o64["score"][ok]) / np.abs(o64["score"][ok])
    re = path_scores(batch, pairs, pair_off, res["n_pairs"], ok)
    gap = o64["score"][ok] - re[ok]
    return {"reads": int(ok.sum()), "near_tie_frac": float(tie[ok].mean()) if ok.any() else None,
            "exact_tie_frac": float(exact[ok].mean()) if ok.any() else None,
            "path_mismatch_non_tie": int(mism), "max_rel_err_fp64": float(rel.max()) if ok.any() else None,
            "max_fp64_gap_of_path": float(np.abs(gap).max()) if ok.any() else None}
