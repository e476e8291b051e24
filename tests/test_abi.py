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


def test_measurement_rows_follow_the_handle_counter(monkeypatch):
    """spin_run measures when the handle's sweep count reaches a multiple of
    measure_every, so the rows a call writes depend on where the counter
    stands: the binding's count (which sizes Lattice.run's series) equals a
    brute-force count of those sweeps."""
    from paper_1101_1427_gb300 import _binding as B
    for cur in range(0, 13):
        monkeypatch.setattr(B, "spin_sweeps_done", lambda h, cur=cur: cur)
        for n in range(0, 11):
            for every in range(0, 5):
                want = sum(1 for s in range(cur + 1, cur + n + 1) if every > 0 and s % every == 0)
                assert B._n_meas(None, n, every) == want, (cur, n, every)


def declared_parameter_counts():
    """Parameter count of every spin_* function declared in include/spin.h."""
    text = open(os.path.join(ROOT, "include", "spin.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(spin_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argtypes_match_the_header():
    """The ctypes signatures of the binding have as many parameters as the
    header's declarations (a drift between the two would pass arguments in
    the wrong places)."""
    from paper_1101_1427_gb300 import _binding as B
    lib = B.lib()
    counts = declared_parameter_counts()
    assert len(counts) == len(declared_symbols())
    bad = {n: (c, len(getattr(lib, n).argtypes)) for n, c in counts.items()
           if len(getattr(lib, n).argtypes or []) != c}
    assert not bad, bad
