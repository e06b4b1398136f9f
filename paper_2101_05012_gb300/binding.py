"""Python binding of libabea (include/abea.h): argument marshalling only.

Every step of the alignment runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors into the pointers and sizes of the C
ABI and back.  It never falls back to a CPU path: if the library cannot be
loaded, load() raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

ABEA_OK = 0
ABEA_ERR_ARG = -1
ABEA_ERR_CAPACITY = -2
ABEA_ERR_NOMEM = -3
ABEA_ERR_CUDA = -4
ABEA_ERR_TIMEOUT = -5
ABEA_ERR_NO_MODEL = -6

READ_OK, READ_FAIL_NO_END, READ_BAD_INPUT, READ_CAPACITY = range(4)
SCALE_OK, SCALE_DEGENERATE, SCALE_BAD_INPUT = range(3)

# the functions include/abea.h declares
EXPORTS = ["abea_create", "abea_destroy", "abea_strerror", "abea_set_model", "abea_align", "abea_align_batch",
           "abea_align_packed", "abea_align_batch_device", "abea_last_launch_stats",
           "abea_set_block_mode", "abea_eventalign", "abea_detect_events", "abea_estimate_scalings", "abea_server_start", "abea_server_submit", "abea_server_poll",
           "abea_server_stop", "abea_align_batch_device_noalloc", "abea_f32_from_i64", "abea_f32_from_f64", "abea_summarise",
           "abea_eventalign_tsv", "abea_summary_tsv", "abea_autotune"]


class Scalings(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_float), ("shift", ctypes.c_float), ("var", ctypes.c_float)]


class Read(ctypes.Structure):
    _fields_ = [("ev_mean", ctypes.c_void_p), ("n_events", ctypes.c_int32), ("seq", ctypes.c_void_p),
                ("seq_len", ctypes.c_int32), ("sc", Scalings)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("max_batch_reads", ctypes.c_int32), ("max_wait_us", ctypes.c_int32),
                ("batches_in_flight", ctypes.c_int32), ("max_requests", ctypes.c_int32),
                ("block_theta", ctypes.c_double), ("short_bases", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_float), ("status", ctypes.c_int32), ("n_pairs", ctypes.c_int32),
                ("e_end", ctypes.c_int32), ("cells", ctypes.c_int64)]


EVENTALIGN_DTYPE = np.dtype([("read", "<i4"), ("event", "<i4"), ("kmer", "<i4"), ("ref_pos", "<i4"),
                             ("ref_rank", "<i4"), ("model_rank", "<i4"), ("level", "<f4"), ("model_mean", "<f4"),
                             ("model_stdv", "<f4"), ("z", "<f4")])

EVENT_DTYPE = np.dtype([("mean", "<f4"), ("stdv", "<f4"), ("start", "<i4"), ("length", "<i4")])

TUNE_DTYPE = np.dtype([("W", "<i4"), ("min_bands", "<i4"), ("max_bands", "<i4"), ("sample_reads", "<i4"),
                       ("reads_per_cta", "<i4"), ("threads_per_band", "<i4"), ("record_words", "<i4"),
                       ("gcups_per_warp", "<f4"), ("gcups_block", "<f4")])

SUMMARY_DTYPE = np.dtype([("read", "<i4"), ("status", "<i4"), ("n_events", "<i4"), ("n_kmers", "<i4"),
                          ("n_pairs", "<i4"), ("first_event", "<i4"), ("last_event", "<i4"),
                          ("events_aligned", "<i4"), ("stays", "<i4"), ("skips", "<i4"), ("score", "<f4"),
                          ("score_per_event", "<f4"), ("flags", "<i4")])
QC_NOT_ALIGNED, QC_TRIMMED, QC_SKIPS, QC_LOW_SCORE = 1, 2, 4, 8

RESULT_DTYPE = np.dtype([("score", "<f4"), ("status", "<i4"), ("n_pairs", "<i4"), ("e_end", "<i4"),
                         ("cells", "<i8")])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(Result) == 24

_lib = None


class AbeaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        name = load().abea_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {name} ({code})")


def load(path: Optional[str] = None):
    """Open libabea.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if path is None and not _build.up_to_date():
        _build.build()
    if not os.path.exists(p):
        raise RuntimeError(f"libabea.so not found at {p}: the CUDA extension is required")
    lib = ctypes.CDLL(p)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.abea_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t]
    lib.abea_destroy.argtypes = [P]
    lib.abea_destroy.restype = None
    lib.abea_strerror.argtypes = [ctypes.c_int]
    lib.abea_strerror.restype = ctypes.c_char_p
    lib.abea_set_model.argtypes = [P, ctypes.c_int, P, P]
    lib.abea_align.argtypes = [P, ctypes.POINTER(Read), ctypes.c_int, ctypes.POINTER(Result), P, i32]
    lib.abea_align_batch.argtypes = [P, P, i32, ctypes.c_int, P, P, P, P]
    lib.abea_align_packed.argtypes = [P, i32, ctypes.c_int, P, P, P, P, P, P, P, P, P]
    lib.abea_align_batch_device.argtypes = [P, i32, ctypes.c_int, P, P, P, P, P, P, P, P, P]
    lib.abea_last_launch_stats.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
    lib.abea_set_block_mode.argtypes = [P, ctypes.c_double]
    lib.abea_estimate_scalings.argtypes = [P, i32, P, P, P, P, P, P, P]
    lib.abea_detect_events.argtypes = [P, i32, P, P, P, ctypes.c_int, ctypes.c_float, P, P, P, P]
    lib.abea_eventalign.argtypes = [P, i32, P, P, P, P, P, P, P, P, P, P, i64, ctypes.c_int, P, P]
    lib.abea_server_start.argtypes = [P, ctypes.POINTER(ServerCfg), ctypes.POINTER(P)]
    lib.abea_server_submit.argtypes = [P, ctypes.POINTER(Read), ctypes.POINTER(i64)]
    lib.abea_server_poll.argtypes = [P, i64, i32, ctypes.POINTER(Result), P, i32, ctypes.POINTER(ctypes.c_double)]
    lib.abea_server_stop.argtypes = [P]
    lib.abea_align_batch_device_noalloc.argtypes = [ctypes.c_int, P, P, i32, ctypes.c_int, P, P, P, P, P, P, P, P, P]
    lib.abea_summarise.argtypes = [P, i32, P, P, P, P, P, P, P]
    lib.abea_autotune.argtypes = [P, ctypes.c_int, i32, P, P, P, P, P, P, i32, ctypes.POINTER(i32)]
    lib.abea_eventalign_tsv.argtypes = [P, i64, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_size_t)]
    lib.abea_summary_tsv.argtypes = [P, i32, ctypes.c_int, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    for f in EXPORTS:
        if f not in ("abea_destroy", "abea_strerror"):
            getattr(lib, f).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != ABEA_OK:
        raise AbeaError(rc, what)


def pair_offsets(n_events: np.ndarray, n_kmers: np.ndarray) -> np.ndarray:
    """Pair capacity n_e + n_k - 1 per read (always enough), as offsets."""
    cap = np.maximum(np.asarray(n_events, np.int64) + np.asarray(n_kmers, np.int64) - 1, 1)
    off = np.zeros(len(cap) + 1, np.int64)
    np.cumsum(cap, out=off[1:])
    return off


class Context:
    """An abea_ctx on one CUDA device."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.abea_create(ctypes.byref(h), device, mem_budget_bytes), "abea_create")
        self.h = h
        self.k = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.abea_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_model(self, k: int, level_mean, level_stdv):
        m = np.ascontiguousarray(level_mean, np.float32)
        s = np.ascontiguousarray(level_stdv, np.float32)
        if m.size != 4 ** k or s.size != 4 ** k:
            raise ValueError("model arrays must hold 4^k entries")
        _check(self.lib.abea_set_model(self.h, k, _p(m), _p(s)), "abea_set_model")
        self.k = k

    def align(self, events, seq, scalings, W: int):
        """One read (abea_align).  Returns (result dict, pairs int32[n,2])."""
        ev = np.ascontiguousarray(events, np.float32)
        sq = np.frombuffer(seq.encode() if isinstance(seq, str) else bytes(seq), np.uint8).copy()
        cap = max(len(ev) + len(sq), 1)
        pairs = np.zeros((cap, 2), np.int32)
        rd = Read(_p(ev).value, len(ev), _p(sq).value, len(sq), Scalings(*[float(v) for v in scalings]))
        res = Result()
        _check(self.lib.abea_align(self.h, ctypes.byref(rd), W, ctypes.byref(res), _p(pairs), cap), "abea_align")
        out = {f: getattr(res, f) for f, _ in Result._fields_}
        return out, pairs[:res.n_pairs].copy() if res.status == READ_OK else pairs[:0]

    def align_batch(self, events_list, seqs, scalings, W: int, stream=None):
        """abea_align_batch over lists of reads.  Returns (results, pairs, pair_off)."""
        n = len(events_list)
        evs = [np.ascontiguousarray(e, np.float32) for e in events_list]
        sqs = [np.frombuffer(s.encode() if isinstance(s, str) else bytes(s), np.uint8).copy() for s in seqs]
        recs = (Read * max(n, 1))()
        for i in range(n):
            sc = scalings[i]
            recs[i] = Read(_p(evs[i]).value if len(evs[i]) else None, len(evs[i]),
                           _p(sqs[i]).value if len(sqs[i]) else None, len(sqs[i]),
                           Scalings(float(sc[0]), float(sc[1]), float(sc[2])))
        n_k = np.array([len(s) for s in sqs], np.int64) - (self.k or 1) + 1
        pair_off = pair_offsets([len(e) for e in evs], np.maximum(n_k, 1))
        out = np.zeros(n, RESULT_DTYPE)
        pairs = np.zeros((max(int(pair_off[-1]), 1), 2), np.int32)
        _check(self.lib.abea_align_batch(self.h, ctypes.cast(recs, ctypes.c_void_p), n, W, _p(out), _p(pairs),
                                         _p(pair_off), ctypes.c_void_p(stream)), "abea_align_batch")
        return out, pairs, pair_off

    def align_packed(self, batch, W: Optional[int] = None, stream=None, pair_off=None):
        """abea_align_packed over a synth.Batch (host arrays).  Returns (results, pairs, pair_off)."""
        W = batch.W if W is None else W
        n = batch.n
        if pair_off is None:
            pair_off = pair_offsets(batch.n_events(), np.maximum(batch.n_kmers(), 1))
        out = np.zeros(n, RESULT_DTYPE)
        pairs = np.zeros((max(int(pair_off[-1]), 1), 2), np.int32)
        sc = np.ascontiguousarray(batch.scalings, np.float32)
        _check(self.lib.abea_align_packed(self.h, n, W, _p(batch.seq), _p(batch.seq_off), _p(batch.events),
                                          _p(batch.ev_off), _p(sc), _p(out), _p(pairs), _p(pair_off),
                                          ctypes.c_void_p(stream)), "abea_align_packed")
        return out, pairs, pair_off

    def align_batch_device(self, n: int, W: int, d_seq, seq_off, d_events, ev_off, scalings, d_out, d_pairs,
                           pair_off, stream=None):
        """abea_align_batch_device: d_* are torch CUDA tensors (uint8 bases, float32 events,
        uint8[n*24] results, int32 pairs); offsets and scalings are host numpy arrays."""
        sc = np.ascontiguousarray(scalings, np.float32)
        so = np.ascontiguousarray(seq_off, np.int64)
        eo = np.ascontiguousarray(ev_off, np.int64)
        po = np.ascontiguousarray(pair_off, np.int64)
        _check(self.lib.abea_align_batch_device(
            self.h, n, W, ctypes.c_void_p(d_seq.data_ptr()), _p(so), ctypes.c_void_p(d_events.data_ptr()), _p(eo),
            _p(sc), ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(d_pairs.data_ptr()), _p(po),
            ctypes.c_void_p(stream)), "abea_align_batch_device")

    def eventalign(self, n: int, d_seq, seq_off, d_events, ev_off, scalings, d_results, d_pairs, pair_off, d_ref_pos,
                   d_ref, ref_len: int, scale_events: bool, d_rows, stream=None):
        """abea_eventalign: d_* are torch CUDA tensors (d_results and d_pairs as filled by
        align_batch_device, d_rows 40 bytes per pair slot); offsets and scalings host arrays."""
        so = np.ascontiguousarray(seq_off, np.int64)
        eo = np.ascontiguousarray(ev_off, np.int64)
        po = np.ascontiguousarray(pair_off, np.int64)
        sc = np.ascontiguousarray(scalings, np.float32)
        _check(self.lib.abea_eventalign(
            self.h, n, ctypes.c_void_p(d_seq.data_ptr()), _p(so), ctypes.c_void_p(d_events.data_ptr()), _p(eo), _p(sc),
            ctypes.c_void_p(d_results.data_ptr()), ctypes.c_void_p(d_pairs.data_ptr()), _p(po),
            ctypes.c_void_p(d_ref_pos.data_ptr()), ctypes.c_void_p(d_ref.data_ptr()), int(ref_len),
            1 if scale_events else 0, ctypes.c_void_p(d_rows.data_ptr()), ctypes.c_void_p(stream)),
            "abea_eventalign")

    def detect_events(self, n: int, d_raw, raw_off, calib, window: int, tau2: float, d_events, event_off, d_n_events,
                      stream=None):
        """abea_detect_events: d_raw int16, d_events (16 bytes per event) and d_n_events int32 are torch
        CUDA tensors; raw_off, calib (float32[n, 2]) and event_off host arrays."""
        ro = np.ascontiguousarray(raw_off, np.int64)
        eo = np.ascontiguousarray(event_off, np.int64)
        ca = np.ascontiguousarray(calib, np.float32)
        _check(self.lib.abea_detect_events(
            self.h, n, ctypes.c_void_p(d_raw.data_ptr()), _p(ro), _p(ca), window, tau2,
            ctypes.c_void_p(d_events.data_ptr()), _p(eo), ctypes.c_void_p(d_n_events.data_ptr()),
            ctypes.c_void_p(stream)), "abea_detect_events")

    def estimate_scalings(self, n: int, d_seq, seq_off, d_events, ev_off, d_out, d_status, stream=None):
        """abea_estimate_scalings: d_* are torch CUDA tensors (uint8 bases, float32 events, float32[n*3]
        scalings out, int32[n] status out); offsets are host numpy arrays."""
        so = np.ascontiguousarray(seq_off, np.int64)
        eo = np.ascontiguousarray(ev_off, np.int64)
        _check(self.lib.abea_estimate_scalings(
            self.h, n, ctypes.c_void_p(d_seq.data_ptr()), _p(so), ctypes.c_void_p(d_events.data_ptr()), _p(eo),
            ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(d_status.data_ptr()), ctypes.c_void_p(stream)),
            "abea_estimate_scalings")

    def summarise(self, n: int, seq_off, ev_off, d_results, d_pairs, pair_off, d_out, stream=None):
        """abea_summarise: d_results and d_pairs as filled by align_batch_device, d_out a torch CUDA
        tensor of n * 52 bytes; offsets are host numpy arrays."""
        so = np.ascontiguousarray(seq_off, np.int64)
        eo = np.ascontiguousarray(ev_off, np.int64)
        po = np.ascontiguousarray(pair_off, np.int64)
        _check(self.lib.abea_summarise(self.h, n, _p(so), _p(eo), ctypes.c_void_p(d_results.data_ptr()),
                                       ctypes.c_void_p(d_pairs.data_ptr()), _p(po), ctypes.c_void_p(d_out.data_ptr()),
                                       ctypes.c_void_p(stream)), "abea_summarise")

    def autotune(self, batch, W: Optional[int] = None) -> np.ndarray:
        """abea_autotune on a synth.Batch sample; returns the choices (TUNE_DTYPE)."""
        W = batch.W if W is None else W
        out = np.zeros(4, TUNE_DTYPE)
        n_out = ctypes.c_int32()
        sc = np.ascontiguousarray(batch.scalings, np.float32)
        _check(self.lib.abea_autotune(self.h, W, batch.n, _p(batch.seq), _p(batch.seq_off), _p(batch.events),
                                      _p(batch.ev_off), _p(sc), _p(out), 4, ctypes.byref(n_out)), "abea_autotune")
        return out[:n_out.value].copy()

    def set_block_mode(self, theta: float):
        """Reads above theta x the even per-warp share of bands run on a whole block (<= 0: never)."""
        _check(self.lib.abea_set_block_mode(self.h, float(theta)), "abea_set_block_mode")

    def last_launch_stats(self):
        n = ctypes.c_int32()
        ms = ctypes.c_float()
        _check(self.lib.abea_last_launch_stats(self.h, ctypes.byref(n), ctypes.byref(ms)), "abea_last_launch_stats")
        return n.value, ms.value


class Server:
    """abea_server_*: continuous admission of single-read requests on a Context's device and model."""

    def __init__(self, ctx: Context, W: int, max_batch_reads: int = 0, max_wait_us: int = 0,
                 batches_in_flight: int = 0, max_requests: int = 0, block_theta: float = 1.0,
                 short_bases: int = 0):
        self.lib = ctx.lib
        self.k = ctx.k
        cfg = ServerCfg(W, max_batch_reads, max_wait_us, batches_in_flight, max_requests, float(block_theta),
                        short_bases)
        h = ctypes.c_void_p()
        _check(self.lib.abea_server_start(ctx.h, ctypes.byref(cfg), ctypes.byref(h)), "abea_server_start")
        self.h = h
        self._keep = {}

    def submit(self, events, seq, scalings) -> int:
        """Queue one read; returns its ticket.  Raises AbeaError (ABEA_ERR_CAPACITY when full)."""
        ev = np.ascontiguousarray(events, np.float32)
        sq = np.frombuffer(seq.encode() if isinstance(seq, str) else bytes(seq), np.uint8).copy()
        rd = Read(_p(ev).value if len(ev) else None, len(ev), _p(sq).value if len(sq) else None, len(sq),
                  Scalings(*[float(v) for v in scalings]))
        t = ctypes.c_int64()
        _check(self.lib.abea_server_submit(self.h, ctypes.byref(rd), ctypes.byref(t)), "abea_server_submit")
        self._keep[t.value] = len(ev) + max(len(sq), 1)
        return t.value

    def poll(self, ticket: int, wait_us: int = 0):
        """(result dict, pairs int32[n,2], latency_us), or None while the request runs."""
        cap = max(self._keep.get(ticket, 1), 1)
        pairs = np.zeros((cap, 2), np.int32)
        res = Result()
        lat = ctypes.c_double()
        rc = self.lib.abea_server_poll(self.h, ticket, wait_us, ctypes.byref(res), _p(pairs), cap,
                                       ctypes.byref(lat))
        if rc == ABEA_ERR_TIMEOUT:
            return None
        _check(rc, "abea_server_poll")
        self._keep.pop(ticket, None)
        out = {f: getattr(res, f) for f, _ in Result._fields_}
        return out, pairs[:res.n_pairs].copy() if res.status == READ_OK else pairs[:0], lat.value

    def stop(self):
        if getattr(self, "h", None):
            self.lib.abea_server_stop(self.h)
            self.h = None

    def __del__(self):
        self.stop()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()


def align_batch_device_noalloc(k: int, level_mean, level_stdv, n: int, W: int, d_seq, seq_off, d_events, ev_off,
                               scalings, d_out, d_pairs, pair_off, stream=None):
    """abea_align_batch_device_noalloc (no context, no allocation): d_* are torch CUDA
    tensors on the current device; model, offsets and scalings are host arrays."""
    lib = load()
    mm = np.ascontiguousarray(level_mean, np.float32)
    ms = np.ascontiguousarray(level_stdv, np.float32)
    sc = np.ascontiguousarray(scalings, np.float32)
    so = np.ascontiguousarray(seq_off, np.int64)
    eo = np.ascontiguousarray(ev_off, np.int64)
    po = np.ascontiguousarray(pair_off, np.int64)
    _check(lib.abea_align_batch_device_noalloc(
        k, _p(mm), _p(ms), n, W, ctypes.c_void_p(d_seq.data_ptr()), _p(so), ctypes.c_void_p(d_events.data_ptr()),
        _p(eo), _p(sc), ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(d_pairs.data_ptr()), _p(po),
        ctypes.c_void_p(stream)), "abea_align_batch_device_noalloc")


def f32_from_i64(d_in, d_out, stream=None):
    """abea_f32_from_i64: d_in int64 and d_out float32 torch CUDA tensors of the same length."""
    lib = load()
    _check(lib.abea_f32_from_i64(ctypes.c_void_p(d_in.data_ptr()), ctypes.c_int64(d_in.numel()),
                                 ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream)), "abea_f32_from_i64")


def f32_from_f64(d_in, d_out, stream=None):
    """abea_f32_from_f64: d_in float64 and d_out float32 torch CUDA tensors of the same length."""
    lib = load()
    _check(lib.abea_f32_from_f64(ctypes.c_void_p(d_in.data_ptr()), ctypes.c_int64(d_in.numel()),
                                 ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream)), "abea_f32_from_f64")


def _text(fn, *args) -> str:
    need = ctypes.c_size_t()
    rc = fn(*args, None, 0, ctypes.byref(need))
    if rc not in (ABEA_OK, ABEA_ERR_CAPACITY):
        _check(rc, fn.__name__)
    buf = ctypes.create_string_buffer(need.value + 1)
    _check(fn(*args, buf, need.value + 1, ctypes.byref(need)), fn.__name__)
    return buf.value.decode()


def eventalign_tsv(rows: np.ndarray, k: int, header: bool = True) -> str:
    """abea_eventalign_tsv over host rows (EVENTALIGN_DTYPE)."""
    r = np.ascontiguousarray(rows, EVENTALIGN_DTYPE)
    return _text(load().abea_eventalign_tsv, _p(r), ctypes.c_int64(len(r)), k, 1 if header else 0)


def summary_tsv(summaries: np.ndarray, header: bool = True) -> str:
    """abea_summary_tsv over host summaries (SUMMARY_DTYPE)."""
    s = np.ascontiguousarray(summaries, SUMMARY_DTYPE)
    return _text(load().abea_summary_tsv, _p(s), len(s), 1 if header else 0)


def results_from_bytes(buf: np.ndarray) -> np.ndarray:
    """View a uint8 buffer of n*24 bytes (device results copied back) as results."""
    return np.frombuffer(np.ascontiguousarray(buf).tobytes(), RESULT_DTYPE)
