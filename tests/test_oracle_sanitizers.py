"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer
(host only): a sanitized build runs single reads in both precisions, the full
DP, the threaded batch driver, rejected inputs, capacity overflow and k-mer
ranks, in a child process with the sanitizer runtimes preloaded; any report
fails the test."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
from oracle import oracle
from paper_2101_05012_gb300 import synth
oracle._lib = oracle._setup(ctypes.CDLL(LIB))
b = synth.make_batch("plain_64x1kb", n_reads=6)
for i in range(3):
    e, s, sc = b.read(i)
    for prec in ("f64", "f32"):
        r = oracle.abea(b.model_mean, b.model_stdv, b.k, s, e, sc, b.W, precision=prec)
        assert r["status"] == oracle.ST_OK, r["status"]
    r = oracle.abea(b.model_mean, b.model_stdv, b.k, s, e, sc, b.W, with_bands=True)
    assert r["status"] == oracle.ST_OK and r["bands"].shape[1] == b.W
# a pair buffer that is too small: the status says so and nothing is written past it
e, s, sc = b.read(3)
lib = oracle._lib
mm = np.ascontiguousarray(b.model_mean, np.float32); ms = np.ascontiguousarray(b.model_stdv, np.float32)
sq = np.frombuffer(bytes(s), np.uint8).copy(); ev = np.ascontiguousarray(e, np.float32)
pairs = np.zeros((5, 2), np.int32); res = oracle.OracleResult()
lib.oracle_abea_f32(oracle._ptr(mm), oracle._ptr(ms), b.k, oracle._ptr(sq), len(sq), oracle._ptr(ev), len(ev),
                    float(sc[0]), float(sc[1]), float(sc[2]), b.W, oracle._ptr(pairs), 5, ctypes.byref(res), None, None)
assert res.status == oracle.ST_CAPACITY, res.status
e, s, sc = b.read(0)
oracle.full_dp(b.model_mean, b.model_stdv, b.k, s[:40], e[:60], sc)
bad = s[:100] + b"N" + s[101:]
assert oracle.abea(b.model_mean, b.model_stdv, b.k, bad, e, sc, b.W)["status"] == oracle.ST_BAD_INPUT
assert oracle.abea(b.model_mean, b.model_stdv, b.k, s, e[:1], sc, b.W)["status"] in (oracle.ST_OK, oracle.ST_FAIL_NO_END)
oracle.abea_batch(b, "f32", n_threads=3)
oracle.kmer_ranks(b"ACGTNACGTTGCA", 4)
oracle.constants(100, 60)
print("sanitized oracle ok")
"""


def test_oracle_under_asan_and_ubsan(tmp_path):
    gcc = "gcc"
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        p = subprocess.run([gcc, f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            pytest.skip(f"{name} not available")
        libs.append(p)
    sys.path.insert(0, ROOT)
    from oracle import oracle
    lib = oracle.build(out=str(tmp_path / "liboracle_san.so"),
                       extra_flags=("-g", "-O1", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                                    "-fno-sanitize-recover=undefined"))
    env = dict(os.environ, LD_PRELOAD=":".join(libs), ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + SCRIPT
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    report = p.stderr[-4000:]
    assert p.returncode == 0, report
    assert "runtime error" not in p.stderr and "AddressSanitizer" not in p.stderr, report
    assert "sanitized oracle ok" in p.stdout
