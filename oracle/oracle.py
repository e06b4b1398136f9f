"""Python access to the CPU oracle of ABEA (oracle/abea_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product path (the CUDA library and its
binding) never imports this module.

`build()` compiles abea_oracle.c twice (FP64, and FP32 with -DORACLE_F32)
with -O3 -ffp-contract=off into oracle/_build/liboracle.so (no fused
multiply-add unless written as fma(), no reassociation: the results do not
depend on the optimisation level or the host; no -march=native, so the same
source gives the same code paths on the x86 and Arm hosts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "abea_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

ST_OK, ST_FAIL_NO_END, ST_BAD_INPUT, ST_CAPACITY, ST_NOMEM, ST_INTERNAL = range(6)
TR_D, TR_U, TR_L = 0, 1, 2


class OracleResult(ctypes.Structure):
    _fields_ = [("score", ctypes.c_double), ("status", ctypes.c_int32), ("n_pairs", ctypes.c_int32),
                ("e_end", ctypes.c_int32), ("cells", ctypes.c_int64), ("min_margin", ctypes.c_double)]


def build(src: str = SRC, out: str = LIB, extra_flags=()) -> str:
    """Compile the oracle (both precisions) into a shared library; returns its path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O3", "-ffp-contract=off", "-fPIC", "-std=c11", "-D_POSIX_C_SOURCE=200809L", *extra_flags]
    o64 = out + ".f64.o"
    o32 = out + ".f32.o"
    subprocess.run(base + ["-c", src, "-o", o64], check=True)
    subprocess.run(base + ["-DORACLE_F32", "-c", src, "-o", o32], check=True)
    subprocess.run(["gcc", "-shared", "-o", out, o64, o32, "-lm", "-lpthread"], check=True)
    return out


_lib = None
_lock = threading.Lock()


def _setup(lib):
    P = ctypes.c_void_p
    i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    for prec in ("f64", "f32"):
        fn = getattr(lib, f"oracle_abea_{prec}")
        fn.argtypes = [P, P, i32, P, i32, P, i32, f32, f32, f32, i32, P, i32,
                       ctypes.POINTER(OracleResult), P, P]
        fn.restype = ctypes.c_int
        fn = getattr(lib, f"oracle_full_dp_{prec}")
        fn.argtypes = [P, P, i32, P, i32, P, i32, f32, f32, f32, P, i32, ctypes.POINTER(OracleResult)]
        fn.restype = ctypes.c_int
        fn = getattr(lib, f"oracle_abea_batch_{prec}")
        fn.argtypes = [P, P, i32, i32, i32, P, P, P, P, P, P, P, P, i32]
        fn.restype = ctypes.c_int
    lib.oracle_kmer_ranks.argtypes = [P, i32, i32, P]
    lib.oracle_kmer_ranks.restype = ctypes.c_int
    lib.oracle_constants.argtypes = [i32, i32, P]
    lib.oracle_constants.restype = None
    return lib


def load(path: Optional[str] = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    with _lock:
        if path is not None:
            return _setup(ctypes.CDLL(path))
        if _lib is None:
            here = os.path.abspath(__file__)
            if (not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)
                    or os.path.getmtime(LIB) < os.path.getmtime(here)):
                build()
            _lib = _setup(ctypes.CDLL(LIB))
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def constants(n_events: int, n_kmers: int, lib=None):
    """(lp_skip, lp_stay, lp_step, lp_trim) in FP64."""
    lib = lib or load()
    out = np.zeros(4, np.float64)
    lib.oracle_constants(n_events, n_kmers, _ptr(out))
    return tuple(float(v) for v in out)


def kmer_ranks(seq, k: int, lib=None) -> Optional[np.ndarray]:
    lib = lib or load()
    s = np.frombuffer(seq.encode() if isinstance(seq, str) else bytes(seq), np.uint8)
    out = np.zeros(max(len(s) - k + 1, 0), np.int32)
    if lib.oracle_kmer_ranks(_ptr(s), len(s), k, _ptr(out)) != 0:
        return None
    return out


def abea(model_mean, model_stdv, k, seq, events, scalings, W, precision="f64",
         with_bands=False, lib=None):
    """Align one read.  Returns a dict with score, status, pairs (n,2), e_end,
    cells, min_margin and, with with_bands, ll (n_bands,2) and bands (n_bands,W)."""
    lib = lib or load()
    mm = np.ascontiguousarray(model_mean, np.float32)
    ms = np.ascontiguousarray(model_stdv, np.float32)
    s = np.frombuffer(seq.encode() if isinstance(seq, str) else bytes(seq), np.uint8).copy()
    ev = np.ascontiguousarray(events, np.float32)
    n_k = len(s) - k + 1
    cap = max(len(ev) + max(n_k, 0), 1)
    pairs = np.zeros((cap, 2), np.int32)
    res = OracleResult()
    ll = bands = None
    if with_bands and n_k >= 1 and len(ev) >= 1:
        nb = len(ev) + n_k + 1
        ll = np.zeros((nb, 2), np.int32)
        bands = np.zeros((nb, W), np.float64 if precision == "f64" else np.float32)
    fn = getattr(lib, f"oracle_abea_{precision}")
    fn(_ptr(mm), _ptr(ms), k, _ptr(s), len(s), _ptr(ev), len(ev),
       float(scalings[0]), float(scalings[1]), float(scalings[2]), W,
       _ptr(pairs), cap, ctypes.byref(res),
       _ptr(ll) if ll is not None else None, _ptr(bands) if bands is not None else None)
    out = dict(score=res.score, status=res.status, pairs=pairs[:res.n_pairs].copy() if res.status == ST_OK else pairs[:0],
               n_pairs=res.n_pairs, e_end=res.e_end, cells=res.cells, min_margin=res.min_margin)
    if with_bands:
        out["ll"] = ll
        out["bands"] = bands
    return out


def full_dp(model_mean, model_stdv, k, seq, events, scalings, precision="f64", lib=None):
    """Unbanded DP of the same recurrence; same output dict as abea()."""
    lib = lib or load()
    mm = np.ascontiguousarray(model_mean, np.float32)
    ms = np.ascontiguousarray(model_stdv, np.float32)
    s = np.frombuffer(seq.encode() if isinstance(seq, str) else bytes(seq), np.uint8).copy()
    ev = np.ascontiguousarray(events, np.float32)
    cap = max(len(ev) + len(s), 1)
    pairs = np.zeros((cap, 2), np.int32)
    res = OracleResult()
    getattr(lib, f"oracle_full_dp_{precision}")(
        _ptr(mm), _ptr(ms), k, _ptr(s), len(s), _ptr(ev), len(ev),
        float(scalings[0]), float(scalings[1]), float(scalings[2]), _ptr(pairs), cap, ctypes.byref(res))
    return dict(score=res.score, status=res.status, pairs=pairs[:res.n_pairs].copy() if res.status == ST_OK else pairs[:0],
                n_pairs=res.n_pairs, e_end=res.e_end, cells=res.cells, min_margin=res.min_margin)


def abea_batch(batch, precision="f32", n_threads: int = 1, W: Optional[int] = None, lib=None):
    """Align every read of a synth.Batch.  Returns dict of arrays:
    score f64[n], status i32[n], n_pairs i32[n], e_end i32[n], cells i64[n],
    min_margin f64[n], pairs i32[P,2], pair_off i64[n+1]."""
    lib = lib or load()
    W = batch.W if W is None else W
    n = batch.n
    cap = (batch.n_events() + np.maximum(batch.n_kmers(), 0)).astype(np.int64)
    pair_off = np.zeros(n + 1, np.int64)
    np.cumsum(cap, out=pair_off[1:])
    pairs = np.zeros((max(int(pair_off[-1]), 1), 2), np.int32)
    res = (OracleResult * max(n, 1))()
    sc = np.ascontiguousarray(batch.scalings, np.float32)
    getattr(lib, f"oracle_abea_batch_{precision}")(
        _ptr(np.ascontiguousarray(batch.model_mean, np.float32)),
        _ptr(np.ascontiguousarray(batch.model_stdv, np.float32)), batch.k, W, n,
        _ptr(batch.seq), _ptr(batch.seq_off), _ptr(batch.events), _ptr(batch.ev_off), _ptr(sc),
        _ptr(pairs), _ptr(pair_off), ctypes.cast(res, ctypes.c_void_p), int(n_threads))
    arr = np.ctypeslib.as_array(ctypes.cast(res, ctypes.POINTER(ctypes.c_byte)), shape=(ctypes.sizeof(res),))
    rec = np.frombuffer(arr.tobytes(), dtype=np.dtype([("score", "<f8"), ("status", "<i4"), ("n_pairs", "<i4"),
                                                       ("e_end", "<i4"), ("pad", "<i4"), ("cells", "<i8"),
                                                       ("min_margin", "<f8")]))[:n]
    return dict(score=rec["score"].copy(), status=rec["status"].copy(), n_pairs=rec["n_pairs"].copy(),
                e_end=rec["e_end"].copy(), cells=rec["cells"].copy(), min_margin=rec["min_margin"].copy(),
                pairs=pairs, pair_off=pair_off)
