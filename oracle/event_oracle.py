"""CPU oracle of event detection (raw signal -> events).

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU-baseline leg.
The product path never imports it.

The thesis (Sec. "Methylation calling") defines event detection as the
segmentation of a read's raw signal at sudden changes of the signal level,
each segment (event) described by the mean, standard deviation and duration
of its samples; it gives no detector.  This module takes a two-window
t-test reading, with every decision taken in integers or in one fixed FP32
order so that another implementation can reproduce it bit for bit:

  For a window length w and a sample position i with w <= i <= n - w, the
  left window is x[i-w:i], the right window x[i:i+w].  With exact integer
  sums S_L, S_R of the samples and Q_L, Q_R of their squares,
      N_i = w * (S_R - S_L)^2,   D_i = w * (Q_L + Q_R) - S_L^2 - S_R^2,
  so that N_i / D_i = (m_R - m_L)^2 / ((v_L + v_R) / w) with population
  means m and variances v: the squared Welch statistic of the two windows.
  t2_i = float32(N_i) / float32(D_i) (IEEE round to nearest), +inf if
  D_i = 0 < N_i, 0 if N_i = 0; t2_i = 0 for the other positions.

  Position i (1 <= i <= n-1) starts a new event when t2_i >= tau2, t2_i is
  larger than t2_j for every j in [i-w+1, i-1] and not smaller than t2_j
  for every j in [i+1, i+w-1] (a local maximum; ties go to the earliest).

  The events are the segments between consecutive starts (and 0, n).  For a
  segment of L samples with exact sums S, Q:
      mean = float32(S) / float32(L),  var = float32(Q) / float32(L) - mean * mean,
      stdv = sqrt(max(var, 0)),
  then in pA with the read's calibration (offset, pA per unit):
      mean_pA = (mean + offset) * per_unit,  stdv_pA = stdv * per_unit,
  every step a single FP32 operation.
"""
from __future__ import annotations

import numpy as np

F = np.float32


def t2_values(raw, w: int) -> np.ndarray:
    x = np.asarray(raw, dtype=np.int64)
    n = len(x)
    t2 = np.zeros(n, dtype=np.float32)
    if n < 2 * w:
        return t2
    S = np.concatenate([[0], np.cumsum(x)])
    Q = np.concatenate([[0], np.cumsum(x * x)])
    i = np.arange(w, n - w + 1)
    SL, SR = S[i] - S[i - w], S[i + w] - S[i]
    QL, QR = Q[i] - Q[i - w], Q[i + w] - Q[i]
    N = w * (SR - SL) ** 2
    D = w * (QL + QR) - SL * SL - SR * SR
    with np.errstate(divide="ignore", invalid="ignore"):
        v = N.astype(np.float32) / D.astype(np.float32)
    v = np.where(D == 0, np.where(N > 0, np.float32(np.inf), np.float32(0.0)), v).astype(np.float32)
    t2[i] = v
    return t2


def boundaries(t2: np.ndarray, w: int, tau2: float) -> np.ndarray:
    """Sample positions that start a new event (excluding 0), ascending."""
    n = len(t2)
    tau2 = F(tau2)
    out = []
    for i in range(1, n):
        v = t2[i]
        if not (v >= tau2):
            continue
        if any(t2[j] >= v for j in range(max(0, i - w + 1), i)):
            continue
        if any(t2[j] > v for j in range(i + 1, min(n, i + w))):
            continue
        out.append(i)
    return np.array(out, dtype=np.int64)


def detect(raw, w: int, tau2: float, calib):
    """Events of one read: (mean_pA float32, stdv_pA float32, start int64, length int64)."""
    x = np.asarray(raw, dtype=np.int64)
    n = len(x)
    if n == 0:
        z = np.zeros(0)
        return z.astype(np.float32), z.astype(np.float32), z.astype(np.int64), z.astype(np.int64)
    b = np.concatenate([[0], boundaries(t2_values(x, w), w, tau2), [n]])
    S = np.concatenate([[0], np.cumsum(x)])
    Q = np.concatenate([[0], np.cumsum(x * x)])
    offset, per_unit = F(calib[0]), F(calib[1])
    means, stdvs = [], []
    for a, c in zip(b[:-1], b[1:]):
        L = F(c - a)
        mean = F(S[c] - S[a]) / L
        var = F(F(Q[c] - Q[a]) / L) - F(mean * mean)
        stdv = np.sqrt(max(var, F(0.0)), dtype=np.float32)
        means.append(F(F(mean + offset) * per_unit))
        stdvs.append(F(stdv * per_unit))
    return (np.array(means, dtype=np.float32), np.array(stdvs, dtype=np.float32), b[:-1].astype(np.int64),
            (b[1:] - b[:-1]).astype(np.int64))


def detect_batch(rb, w: int, tau2: float):
    """Per read detect() over a synth.RawBatch: (means, stdvs, starts, lengths, offsets)."""
    ms, ss, st, ln, cnt = [], [], [], [], [0]
    for i in range(rb.n):
        m, s, a, L = detect(rb.signal(i), w, tau2, rb.calib[i])
        ms.append(m)
        ss.append(s)
        st.append(a)
        ln.append(L)
        cnt.append(cnt[-1] + len(m))
    cat = lambda v, t: np.concatenate(v).astype(t) if v else np.zeros(0, t)
    return (cat(ms, np.float32), cat(ss, np.float32), cat(st, np.int64), cat(ln, np.int64),
            np.array(cnt, dtype=np.int64))
