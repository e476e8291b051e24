"""The C-ABI library loads and exports every entry point that
include/spin.h declares (no compute: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "spin.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spin_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1101_1427_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert "spin_init" in names and "spin_sweep" in names and len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1101_1427_gb300 import _binding
    missing = [n for n in declared_symbols() if not hasattr(_binding, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_1101_1427_gb300 import _binding as B
    assert B.strerror(B.SPIN_EINVAL) == "invalid argument"
    assert B.strerror(B.SPIN_ETIMEOUT) == "device-side wait timed out"
