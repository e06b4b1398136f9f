"""CPU oracle of the per-read scaling estimate (method of moments).

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU-baseline leg.
The product path never imports it.

The thesis (Sec. "Read-model scaling") says that shift and scale are
estimated per read before ABEA with a method of moments, and that the model
means are then scaled as mu * scale + shift; it gives no formula.  This
module takes the plain reading: match the first two moments of the read's
event means to those of the model level means along the read's k-mer
sequence.  With population moments (divide by the count)

    m_e = mean(x_i),  v_e = mean((x_i - m_e)^2)         over the n_e events
    m_m = mean(mu_r), v_m = mean((mu_r - m_m)^2)         over the n_k k-mers r
    scale = sqrt(v_e / v_m),  shift = m_e - scale * m_m,  var = 1

so that mu * scale + shift has the events' mean and variance.  A read with
fewer than two events, or with v_e = 0 or v_m = 0, is degenerate: scale = 1,
shift = m_e - m_m.  A read with no event, no k-mer, a base outside ACGT or a
non-finite event is rejected.  Everything is FP64, two passes, in the order
written above.
"""
from __future__ import annotations

import numpy as np

from . import oracle

SC_OK, SC_DEGENERATE, SC_BAD_INPUT = 0, 1, 2


def estimate(model_mean, k: int, seq, events):
    """(scale, shift, status) of one read."""
    ev = np.asarray(events, dtype=np.float64)
    ranks = oracle.kmer_ranks(seq, k)
    if ranks is None or len(ranks) < 1 or len(ev) < 1 or not np.all(np.isfinite(ev)):
        return 1.0, 0.0, SC_BAD_INPUT
    mu = np.asarray(model_mean, dtype=np.float64)[ranks]
    m_e = ev.sum() / len(ev)
    m_m = mu.sum() / len(mu)
    v_e = ((ev - m_e) ** 2).sum() / len(ev)
    v_m = ((mu - m_m) ** 2).sum() / len(mu)
    if len(ev) < 2 or v_e == 0.0 or v_m == 0.0:
        return 1.0, m_e - m_m, SC_DEGENERATE
    scale = np.sqrt(v_e / v_m)
    return float(scale), float(m_e - scale * m_m), SC_OK


def estimate_batch(batch):
    """Per-read (scale, shift, status) arrays of a synth.Batch."""
    n = batch.n
    scale = np.zeros(n)
    shift = np.zeros(n)
    status = np.zeros(n, np.int32)
    for i in range(n):
        e, s, _ = batch.read(i)
        scale[i], shift[i], status[i] = estimate(batch.model_mean, batch.k, s, e)
    return scale, shift, status
