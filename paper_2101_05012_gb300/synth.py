"""Seeded synthetic ABEA workloads (inputs only).

This module draws the inputs of Adaptive Banded Event Alignment: a k-mer pore
model, read sequences, per-read scalings and detected events.  It holds none
of the alignment's arithmetic; both the CUDA path and the CPU oracle consume
the arrays it returns.

The workloads stand in for the thesis's nanopore datasets (Ch.5, "Experimental
setup": NA12878 and T778 runs), which are not available.  Their shapes follow
the thesis's description of nanopore data: a pore model of 4^k k-mers with a
mean level and a standard deviation each (Sec. "Methylation calling"), events
that over-segment the k-mers (about 1.5-2.5 events per k-mer, same section and
Sec. "Heuristic based memory pre-allocation"), and a per-read shift/scale of
the model (Sec. "Adaptive Banded Event Alignment", read-model scaling).

Random numbers come from a counter-based generator: the splitmix64 finaliser
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to (seed, stream, counter).  Any element of any read can
therefore be regenerated on its own, and nothing depends on numpy's own
generators, whose streams may change between versions.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags
_T_LEN, _T_ULTRA, _T_SEQ, _T_SKIP, _T_DWELL, _T_NOISE, _T_SCALE, _T_MODEL, _T_ARRIVAL, _T_CLASS = range(1, 11)
_T_RAW_DWELL, _T_RAW_NOISE, _T_CALIB, _T_REF = range(11, 15)

BASES = np.frombuffer(b"ACGT", dtype=np.uint8)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int, sub: int = 0) -> np.uint64:
    """Key of one independent stream (seed, tag, sub)."""
    with np.errstate(over="ignore"):
        a = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) * _GOLDEN + np.uint64(tag))
        b = _mix(a + np.uint64(sub & 0xFFFFFFFFFFFFFFFF) * _GOLDEN)
    return b[0]


def draw_u64(key, idx) -> np.ndarray:
    """The idx-th 64-bit draw of the stream `key` (idx: int or int array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + (idx + np.uint64(1)) * _GOLDEN)


def draw_unit(key, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) (53 random bits)."""
    return (draw_u64(key, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def draw_open_unit(key, idx) -> np.ndarray:
    """Uniform doubles in (0, 1): never 0, so ln() is finite."""
    return ((draw_u64(key, idx) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def draw_normal(key, idx) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of draws 2i, 2i+1."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = draw_open_unit(key, idx * np.uint64(2))
    u2 = draw_unit(key, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass(frozen=True)
class Workload:
    """Recipe of one synthetic workload.

    length: ("fixed", L) or ("lognormal", median, sigma_ln, lo, hi) where hi may be None.
    """
    name: str
    n_reads: int
    k: int
    W: int
    seed: int
    length: tuple
    ultra_frac: float = 0.0
    ultra_range: tuple = (50_000, 200_000)
    dwell_mean: float = 1.8
    skip_prob: float = 0.05
    level_mean_range: tuple = (60.0, 130.0)
    level_stdv_range: tuple = (1.0, 3.0)
    scale_range: tuple = (0.9, 1.1)
    shift_range: tuple = (-5.0, 5.0)
    var_range: tuple = (1.0, 1.5)


# The five workloads: a plain small batch, the one-launch batch, the large
# memory-admitted run, the serving mix (its request classes are drawn by
# `serving_requests`) and the wide k=9 / W=200 model.
WORKLOADS = {
    "plain_64x1kb": Workload("plain_64x1kb", 64, 6, 100, 0, ("fixed", 1000)),
    "batch_4096_ln5kb": Workload("batch_4096_ln5kb", 4096, 6, 100, 1,
                                 ("lognormal", 5000, 0.8, 500, 50_000)),
    "large_50k_ln8kb": Workload("large_50k_ln8kb", 50_000, 6, 100, 2,
                                ("lognormal", 8000, 0.5, 500, None), ultra_frac=0.01),
    "serve_mix": Workload("serve_mix", 4096, 6, 100, 3, ("lognormal", 8000, 0.5, 500, None)),
    "wide_10k_ln10kb_k9_w200": Workload("wide_10k_ln10kb_k9_w200", 10_000, 9, 200, 4,
                                        ("lognormal", 10_000, 0.5, 500, None),
                                        dwell_mean=2.5 / 0.95),
}


@dataclasses.dataclass
class Batch:
    """Packed inputs of a batch of reads (structure of arrays).

    seq      uint8[sum L]   bases 'A','C','G','T' of all reads, concatenated
    seq_off  int64[n+1]     read i is seq[seq_off[i]:seq_off[i+1]]
    events   float32[sum n_e] event means (pA), concatenated
    ev_off   int64[n+1]
    scalings float32[n,3]   (scale, shift, var) per read
    model_mean, model_stdv float32[4^k]
    """
    k: int
    W: int
    model_mean: np.ndarray
    model_stdv: np.ndarray
    seq: np.ndarray
    seq_off: np.ndarray
    events: np.ndarray
    ev_off: np.ndarray
    scalings: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return len(self.seq_off) - 1

    def n_events(self) -> np.ndarray:
        return np.diff(self.ev_off)

    def n_kmers(self) -> np.ndarray:
        return np.diff(self.seq_off) - self.k + 1

    def read(self, i: int):
        """(events, seq bytes, (scale, shift, var)) of read i."""
        ev = self.events[self.ev_off[i]:self.ev_off[i + 1]]
        sq = self.seq[self.seq_off[i]:self.seq_off[i + 1]].tobytes()
        return ev, sq, tuple(float(v) for v in self.scalings[i])

    def subset(self, idx) -> "Batch":
        """A new batch holding reads `idx` (in that order)."""
        idx = np.asarray(idx, dtype=np.int64)
        seqs = [self.seq[self.seq_off[i]:self.seq_off[i + 1]] for i in idx]
        evs = [self.events[self.ev_off[i]:self.ev_off[i + 1]] for i in idx]
        return Batch(self.k, self.W, self.model_mean, self.model_stdv,
                     np.concatenate(seqs) if seqs else np.zeros(0, np.uint8),
                     _offsets([len(s) for s in seqs]),
                     np.concatenate(evs) if evs else np.zeros(0, np.float32),
                     _offsets([len(e) for e in evs]),
                     self.scalings[idx].copy(), self.name)


def _offsets(lengths) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lengths, dtype=np.int64), out=off[1:])
    return off


def make_model(k: int, seed: int, mean_range=(60.0, 130.0), stdv_range=(1.0, 3.0)):
    """Pore model: level_mean ~ U(mean_range), level_stdv ~ U(stdv_range) for all 4^k k-mers."""
    n = 4 ** k
    key = stream_key(seed, _T_MODEL)
    idx = np.arange(n, dtype=np.uint64)
    mean = mean_range[0] + (mean_range[1] - mean_range[0]) * draw_unit(key, 2 * idx)
    stdv = stdv_range[0] + (stdv_range[1] - stdv_range[0]) * draw_unit(key, 2 * idx + np.uint64(1))
    return mean.astype(np.float32), stdv.astype(np.float32)


def read_lengths(w: Workload) -> np.ndarray:
    """Read lengths of a workload (bases)."""
    r = np.arange(w.n_reads, dtype=np.uint64)
    if w.length[0] == "fixed":
        L = np.full(w.n_reads, int(w.length[1]), dtype=np.int64)
    else:
        _, median, sigma, lo, hi = w.length
        z = draw_normal(stream_key(w.seed, _T_LEN), r)
        L = np.rint(median * np.exp(sigma * z)).astype(np.int64)
        L = np.maximum(L, lo)
        if hi is not None:
            L = np.minimum(L, hi)
    if w.ultra_frac > 0:
        u = draw_unit(stream_key(w.seed, _T_ULTRA), 2 * r)
        v = draw_unit(stream_key(w.seed, _T_ULTRA), 2 * r + np.uint64(1))
        lo, hi = np.log(w.ultra_range[0]), np.log(w.ultra_range[1])
        ultra = np.rint(np.exp(lo + (hi - lo) * v)).astype(np.int64)
        L = np.where(u < w.ultra_frac, ultra, L)
    return np.maximum(L, w.k)


def kmer_model_index(codes: np.ndarray, k: int) -> np.ndarray:
    """Model-table row of every k-mer of a base-code array (codes 0..3 = A,C,G,T).

    The table is ordered lexicographically with the first base most
    significant; this is the layout convention of the model arrays.
    """
    n_k = len(codes) - k + 1
    idx = np.zeros(n_k, dtype=np.int64)
    for t in range(k):
        idx = idx * 4 + codes[t:t + n_k]
    return idx


def make_read(w: Workload, r: int, L: int, model_mean, model_stdv, dwell_mean=None,
              prefix: Optional[int] = None):
    """Bases, events and scalings of read r (length L).

    Events walk the k-mers: a k-mer gets no event with probability skip_prob,
    otherwise a geometric number of events on {1,2,...} with mean dwell_mean.
    Each event level is scale*mean + shift + N(0, (stdv*var)^2) for its
    k-mer's model entry.  With `prefix`, only the first `prefix` bases of the
    read (and their events) are kept.
    """
    k = w.k
    dwell_mean = w.dwell_mean if dwell_mean is None else dwell_mean
    kseq = stream_key(w.seed, _T_SEQ, r)
    words = draw_u64(kseq, np.arange((L + 31) // 32, dtype=np.uint64))
    shifts = (np.arange(32, dtype=np.uint64) * np.uint64(2))
    codes = ((words[:, None] >> shifts[None, :]) & np.uint64(3)).reshape(-1)[:L].astype(np.int64)
    if prefix is not None:
        codes = codes[:max(prefix, k)]
    seq = BASES[codes]
    rows = kmer_model_index(codes, k)
    n_k = len(rows)

    ks = stream_key(w.seed, _T_SCALE, r)
    u = draw_unit(ks, np.arange(3, dtype=np.uint64))
    scale = w.scale_range[0] + (w.scale_range[1] - w.scale_range[0]) * u[0]
    shift = w.shift_range[0] + (w.shift_range[1] - w.shift_range[0]) * u[1]
    var = w.var_range[0] + (w.var_range[1] - w.var_range[0]) * u[2]

    j = np.arange(n_k, dtype=np.uint64)
    skip = draw_unit(stream_key(w.seed, _T_SKIP, r), j) < w.skip_prob
    p = 1.0 / dwell_mean
    ud = draw_open_unit(stream_key(w.seed, _T_DWELL, r), j)
    dwell = 1 + np.floor(np.log(ud) / np.log1p(-p)).astype(np.int64)
    dwell[skip] = 0
    if dwell.sum() == 0:
        dwell[0] = 1
    ev_rows = np.repeat(rows, dwell)
    z = draw_normal(stream_key(w.seed, _T_NOISE, r), np.arange(len(ev_rows), dtype=np.uint64))
    mu = model_mean[ev_rows].astype(np.float64)
    sd = model_stdv[ev_rows].astype(np.float64)
    ev = (scale * mu + shift + z * sd * var).astype(np.float32)
    return seq, ev, np.array([scale, shift, var], dtype=np.float32)


def _make_reads(w: Workload, ids, L, mm, ms):
    """Packed bases, base counts, events, event counts and scalings of reads `ids`."""
    seqs, evs, scs = [], [], []
    for r in ids:
        s, e, sc = make_read(w, int(r), int(L[r]), mm, ms)
        seqs.append(s)
        evs.append(e)
        scs.append(sc)
    return (np.concatenate(seqs) if seqs else np.zeros(0, np.uint8), np.array([len(s) for s in seqs], np.int64),
            np.concatenate(evs) if evs else np.zeros(0, np.float32), np.array([len(e) for e in evs], np.int64),
            np.stack(scs) if scs else np.zeros((0, 3), np.float32))


def _make_reads_job(args):
    w, ids = args
    mm, ms = make_model(w.k, w.seed, w.level_mean_range, w.level_stdv_range)
    return _make_reads(w, ids, read_lengths(w), mm, ms)


def make_batch(w, n_reads: Optional[int] = None, read_ids=None, workers: int = 1) -> Batch:
    """Generate a workload (or the first n_reads / the listed reads of it).

    With workers > 1 the reads are generated in that many processes (started
    with "spawn", so the caller may already use CUDA); every read is drawn
    from its own counter-based streams, so the batch is the same either way.
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    mm, ms = make_model(w.k, w.seed, w.level_mean_range, w.level_stdv_range)
    L = read_lengths(w)
    if read_ids is None:
        read_ids = range(w.n_reads if n_reads is None else min(n_reads, w.n_reads))
    ids = np.asarray(list(read_ids), dtype=np.int64)
    if workers > 1 and len(ids) > 4 * workers:
        import multiprocessing as mp
        chunks = [c for c in np.array_split(ids, 4 * workers) if len(c)]
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_make_reads_job, [(w, c) for c in chunks])
    else:
        parts = [_make_reads(w, ids, L, mm, ms)]
    seq = np.concatenate([p[0] for p in parts])
    events = np.concatenate([p[2] for p in parts])
    return Batch(w.k, w.W, mm, ms, seq, _offsets(np.concatenate([p[1] for p in parts])),
                 events, _offsets(np.concatenate([p[3] for p in parts])),
                 np.concatenate([p[4] for p in parts]).reshape(-1, 3), w.name)


def serving_requests(n_requests: int, load: float = 1.0, w: Optional[Workload] = None,
                     channels: int = 512, bases_per_s: float = 450.0,
                     prefix_frac: float = 0.7, prefix_bases: int = 400):
    """Serving mix: Poisson arrivals of read prefixes and full reads.

    The offered load is channels * bases_per_s bases/s times `load`.  A
    request is a 400-base read prefix with probability prefix_frac, else a
    full read of the workload's length distribution.  Returns
    (batch, arrival_s float64[n], is_prefix bool[n]).
    """
    w = WORKLOADS["serve_mix"] if w is None else w
    mm, ms = make_model(w.k, w.seed, w.level_mean_range, w.level_stdv_range)
    wl = dataclasses.replace(w, n_reads=n_requests)
    L = read_lengths(wl)
    is_prefix = draw_unit(stream_key(w.seed, _T_CLASS), np.arange(n_requests, dtype=np.uint64)) < prefix_frac
    seqs, evs, scs = [], [], []
    for r in range(n_requests):
        s, e, sc = make_read(wl, r, int(L[r]), mm, ms, prefix=prefix_bases if is_prefix[r] else None)
        seqs.append(s)
        evs.append(e)
        scs.append(sc)
    mean_bases = prefix_frac * prefix_bases + (1 - prefix_frac) * float(np.mean(L))
    lam = load * channels * bases_per_s / mean_bases
    gaps = -np.log(draw_open_unit(stream_key(w.seed, _T_ARRIVAL), np.arange(n_requests, dtype=np.uint64))) / lam
    batch = Batch(w.k, w.W, mm, ms, np.concatenate(seqs), _offsets([len(s) for s in seqs]),
                  np.concatenate(evs), _offsets([len(e) for e in evs]), np.stack(scs), "serve_mix")
    return batch, np.cumsum(gaps), is_prefix


def custom_batch(events_list, seqs, scalings, model_mean, model_stdv, k, W, name="custom") -> Batch:
    """Pack explicit reads (lists of event arrays, base strings/bytes, scalings)."""
    sq = [np.frombuffer(s.encode() if isinstance(s, str) else bytes(s), dtype=np.uint8) for s in seqs]
    ev = [np.asarray(e, dtype=np.float32) for e in events_list]
    return Batch(k, W, np.asarray(model_mean, np.float32), np.asarray(model_stdv, np.float32),
                 np.concatenate(sq) if sq else np.zeros(0, np.uint8), _offsets([len(s) for s in sq]),
                 np.concatenate(ev) if ev else np.zeros(0, np.float32), _offsets([len(e) for e in ev]),
                 np.asarray(scalings, dtype=np.float32).reshape(-1, 3), name)


@dataclasses.dataclass
class RawBatch:
    """Raw signals of a batch (the input of event detection), packed.

    raw: int16 ADC samples of all reads; read i is raw[raw_off[i]:raw_off[i+1]].
    calib: float32[n, 2] = (offset, pA per ADC unit): pA = (raw + offset) * calib[:, 1].
    starts: the true first sample of each k-mer of each read, packed like
    start_off (for tests of the detector against the generator).
    """
    k: int
    model_mean: np.ndarray
    model_stdv: np.ndarray
    seq: np.ndarray
    seq_off: np.ndarray
    raw: np.ndarray
    raw_off: np.ndarray
    calib: np.ndarray
    starts: np.ndarray
    start_off: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return len(self.raw_off) - 1

    def signal(self, i: int) -> np.ndarray:
        return self.raw[self.raw_off[i]:self.raw_off[i + 1]]


def make_raw_read(w: Workload, r: int, L: int, model_mean, model_stdv, samples_per_base: float = 4000.0 / 450.0):
    """Bases, raw int16 signal, calibration and true k-mer starts of read r.

    The read's bases and scalings are those of make_read.  Each k-mer holds
    the pore for a geometric number of samples (mean samples_per_base, at
    least one); every sample is scale*mean + shift + N(0, (stdv*var)^2) pA of
    its k-mer, digitised as round(pA / pA_per_unit - offset) with a per-read
    offset ~ U(-10, 10) and pA_per_unit = range / 8192, range ~ U(1350, 1450).
    """
    k = w.k
    kseq = stream_key(w.seed, _T_SEQ, r)
    words = draw_u64(kseq, np.arange((L + 31) // 32, dtype=np.uint64))
    shifts = (np.arange(32, dtype=np.uint64) * np.uint64(2))
    codes = ((words[:, None] >> shifts[None, :]) & np.uint64(3)).reshape(-1)[:L].astype(np.int64)
    seq = BASES[codes]
    rows = kmer_model_index(codes, k)
    n_k = len(rows)
    u = draw_unit(stream_key(w.seed, _T_SCALE, r), np.arange(3, dtype=np.uint64))
    scale = w.scale_range[0] + (w.scale_range[1] - w.scale_range[0]) * u[0]
    shift = w.shift_range[0] + (w.shift_range[1] - w.shift_range[0]) * u[1]
    var = w.var_range[0] + (w.var_range[1] - w.var_range[0]) * u[2]
    p = 1.0 / samples_per_base
    ud = draw_open_unit(stream_key(w.seed, _T_RAW_DWELL, r), np.arange(n_k, dtype=np.uint64))
    dwell = 1 + np.floor(np.log(ud) / np.log1p(-p)).astype(np.int64)
    srows = np.repeat(rows, dwell)
    z = draw_normal(stream_key(w.seed, _T_RAW_NOISE, r), np.arange(len(srows), dtype=np.uint64))
    pa = scale * model_mean[srows].astype(np.float64) + shift + z * model_stdv[srows].astype(np.float64) * var
    c = draw_unit(stream_key(w.seed, _T_CALIB, r), np.arange(2, dtype=np.uint64))
    offset = -10.0 + 20.0 * c[0]
    per_unit = (1350.0 + 100.0 * c[1]) / 8192.0
    raw = np.clip(np.rint(pa / per_unit - offset), -32768, 32767).astype(np.int16)
    starts = np.concatenate([[0], np.cumsum(dwell)[:-1]]).astype(np.int64)
    return seq, raw, np.array([offset, per_unit], dtype=np.float32), starts


def make_raw_batch(w, n_reads: Optional[int] = None, read_ids=None) -> RawBatch:
    """Raw signals of a workload's reads (its lengths, model and seed)."""
    w = WORKLOADS[w] if isinstance(w, str) else w
    mm, ms = make_model(w.k, w.seed, w.level_mean_range, w.level_stdv_range)
    L = read_lengths(w)
    ids = np.arange(w.n_reads if n_reads is None else n_reads) if read_ids is None else np.asarray(read_ids)
    seqs, raws, cals, sts = [], [], [], []
    for r in ids:
        s, x, c, st = make_raw_read(w, int(r), int(L[r]), mm, ms)
        seqs.append(s)
        raws.append(x)
        cals.append(c)
        sts.append(st)
    return RawBatch(w.k, mm, ms, np.concatenate(seqs), _offsets([len(x) for x in seqs]),
                    np.concatenate(raws), _offsets([len(x) for x in raws]), np.stack(cals),
                    np.concatenate(sts), _offsets([len(x) for x in sts]), w.name)


def make_ref_alignment(seq, seed: int, r: int, indel_rate: float = 0.03):
    """A reference around a read and the read's base-space alignment to it.

    The reference is the read's bases with indels: at each read base, with
    probability indel_rate/2 the base is missing from the reference (the read
    base is an insertion, aligned to no reference position) and with
    probability indel_rate/2 one random base is inserted into the reference
    before it.  Returns (ref bytes, ref_pos int32[len(seq)]): the reference
    position of each read base, -1 for inserted read bases.
    """
    s = np.frombuffer(seq.encode() if isinstance(seq, str) else bytes(seq), np.uint8)
    n = len(s)
    u = draw_unit(stream_key(seed, _T_REF, r), np.arange(2 * n, dtype=np.uint64))
    drop = u[:n] < indel_rate / 2
    ins = (u[:n] >= indel_rate / 2) & (u[:n] < indel_rate)
    extra = BASES[(draw_u64(stream_key(seed, _T_REF, r), np.arange(2 * n, 3 * n, dtype=np.uint64))
                   & np.uint64(3)).astype(np.int64)]
    ins_n = ins.astype(np.int64)
    keep = (~drop).astype(np.int64)
    start = np.concatenate([[0], np.cumsum(ins_n + keep)[:-1]])     # reference index of read base i's slot
    ref = np.zeros(int((ins_n + keep).sum()), np.uint8)
    ref[start[ins]] = extra[ins]
    pos = np.where(drop, -1, start + ins_n).astype(np.int32)
    ref[pos[~drop]] = s[~drop]
    return ref, pos

