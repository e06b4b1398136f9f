"""CPU oracle of eventalign rows (ABEA pairs -> per-event records).

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU-baseline leg.
The product path never imports it.

The thesis lists `eventalign` as aligning a read's events to reference
k-mers (f5c's command line, with --scale-events: "scale events to the model,
rather than vice-versa") and gives no record format.  This module takes the
plain reading: one row per aligned (event e, read k-mer j) pair of ABEA,
    read, e, j,
    ref_pos  = the reference position of k-mer j's first base through the
               read's base-space alignment (-1 if that base is an insertion),
    ref_rank = the rank of the reference k-mer ref[ref_pos : ref_pos+k]
               (-1 if unaligned, past the reference end or not ACGT),
    model_rank = the rank of read k-mer j,
    level, model_mean, model_stdv, z = (level - model_mean) / model_stdv,
where by default level = x_e, model_mean = mu * scale + shift,
model_stdv = sigma * var; with scale_events, level = (x_e - shift) / scale,
model_mean = mu, model_stdv = sigma * var / scale (z is the same quantity).
All arithmetic is FP32, one operation at a time in the order written.
"""
from __future__ import annotations

import numpy as np

from . import oracle

F = np.float32

ROW_DTYPE = np.dtype([("read", "<i4"), ("event", "<i4"), ("kmer", "<i4"), ("ref_pos", "<i4"),
                      ("ref_rank", "<i4"), ("model_rank", "<i4"), ("level", "<f4"), ("model_mean", "<f4"),
                      ("model_stdv", "<f4"), ("z", "<f4")])


def rows(read: int, model_mean, model_stdv, k: int, seq, events, scalings, pairs, ref, ref_pos,
         scale_events: bool = False) -> np.ndarray:
    ranks = oracle.kmer_ranks(seq, k)
    ref = np.frombuffer(bytes(ref), np.uint8) if not isinstance(ref, np.ndarray) else ref
    scale, shift, var = F(scalings[0]), F(scalings[1]), F(scalings[2])
    out = np.zeros(len(pairs), ROW_DTYPE)
    for t, (e, j) in enumerate(np.asarray(pairs).reshape(-1, 2)):
        x = F(events[e])
        mr = int(ranks[j])
        mu, sd = F(model_mean[mr]), F(model_stdv[mr])
        if scale_events:
            level, mean, stdv = F(F(x - shift) / scale), mu, F(F(sd * var) / scale)
        else:
            level, mean, stdv = x, F(F(mu * scale) + shift), F(sd * var)
        z = F(F(level - mean) / stdv)
        rp = int(ref_pos[j])
        rr = -1
        if rp >= 0 and rp + k <= len(ref):
            r = oracle.kmer_ranks(ref[rp:rp + k].tobytes(), k)
            rr = int(r[0]) if r is not None and len(r) else -1
        out[t] = (read, e, j, rp, rr, mr, level, mean, stdv, z)
    return out


SUMMARY_DTYPE = np.dtype([("read", "<i4"), ("status", "<i4"), ("n_events", "<i4"), ("n_kmers", "<i4"),
                          ("n_pairs", "<i4"), ("first_event", "<i4"), ("last_event", "<i4"),
                          ("events_aligned", "<i4"), ("stays", "<i4"), ("skips", "<i4"), ("score", "<f4"),
                          ("score_per_event", "<f4"), ("flags", "<i4")])
QC_NOT_ALIGNED, QC_TRIMMED, QC_SKIPS, QC_LOW_SCORE = 1, 2, 4, 8


def read_summary(read: int, n_events: int, n_kmers: int, status: int, score, pairs) -> np.ndarray:
    """Summary of one read's alignment (reading of f5c's eventalign --summary, which the thesis only
    names): a walk over its pairs counting stays (next event, same k-mer) and skips (same event, next
    k-mer); trimmed events before the first and after the last pair; FP32 score per event; the quality
    flags NOT_ALIGNED (no alignment), TRIMMED (more than half of the events trimmed), SKIPS (skips
    above a fifth of the k-mers), LOW_SCORE (score per event below -10)."""
    p = np.asarray(pairs).reshape(-1, 2) if status == 0 else np.zeros((0, 2), np.int32)
    stays = skips = 0
    for t in range(1, len(p)):
        de, dk = int(p[t, 0] - p[t - 1, 0]), int(p[t, 1] - p[t - 1, 1])
        if (de, dk) == (1, 0):
            stays += 1
        elif (de, dk) == (0, 1):
            skips += 1
    first = int(p[0, 0]) if len(p) else -1
    last = int(p[-1, 0]) if len(p) else -1
    score = F(score)
    spe = F(score / F(n_events)) if n_events > 0 else F(0)
    if status != 0:
        flags = QC_NOT_ALIGNED
    else:
        flags = 0
        if first + (n_events - 1 - last) > n_events / 2:
            flags |= QC_TRIMMED
        if skips > n_kmers / 5:
            flags |= QC_SKIPS
        if spe < F(-10):
            flags |= QC_LOW_SCORE
    out = np.zeros(1, SUMMARY_DTYPE)
    out[0] = (read, status, n_events, n_kmers, len(p), first, last, len(p) - skips, stays, skips, score, spe, flags)
    return out
