"""The C ABI library builds for sm_103a, loads, and exports every call
include/abea.h declares (no GPU: no compute call is made)."""
import ctypes
import os
import re

from paper_2101_05012_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "abea.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(abea_[a-z0-9_]+)\s*\(", src)))


def test_header_matches_binding():
    assert declared_functions() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the one call that needs no device
    assert lib.abea_strerror(binding.ABEA_ERR_NOMEM) == b"out of memory or memory budget too small"


def test_structs_match_header_layout():
    assert ctypes.sizeof(binding.Result) == 24
    assert ctypes.sizeof(binding.Scalings) == 12
    assert ctypes.sizeof(binding.Read) == 40


def test_built_for_sm103a():
    assert os.path.exists(build.LIB)
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
