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
