"""include/spin.h as a C user sees it: a plain C11 program (tests/c/abi_check.c)
is compiled with gcc -Wall -Wextra -Werror -pedantic against the header and
linked with libspin_gb300.so.  Without a GPU it must build and print the
library's error strings; on a GPU it runs init -> sweep -> measure, whose
lattice, energy and magnetisation must equal the oracle's, and an exchange
run with configuration labels."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    from paper_1101_1427_gb300 import build
    lib = build.build()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    out = str(tmp_path_factory.mktemp("cabi") / "abi_check")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-o", out,
           "-L", libdir, "-lspin_gb300", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _run(program, *args):
    r = subprocess.run([program, *map(str, args)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return r.stdout


def test_c_program_builds_and_reads_error_strings(program):
    from paper_1101_1427_gb300 import _binding as B
    lines = _run(program, "strerror").strip().splitlines()
    got = {int(l.split(" ", 1)[0]): l.split(" ", 1)[1] for l in lines}
    assert set(got) == {0, -1, -2, -3, -4, -5}
    for code, msg in got.items():
        assert msg == B.strerror(code)


@pytest.mark.gpu
def test_c_program_sweep_matches_oracle(program):
    import oracle
    L, n, seed, beta = 32, 9, 77, 0.4407
    out = dict(l.split(" ", 1) for l in _run(program, "ising", L, n, seed, beta).strip().splitlines())
    s = oracle.ising_init(2, L, seed, oracle.lattice_id(0, 0, 0))
    E, M, _ = oracle.ising_run(2, L, s, beta, seed, oracle.lattice_id(0, 0, 0), 0, n)
    assert int(out["SWEEPS"]) == n
    assert int(out["E"]) == E[-1] and int(out["M"]) == M[-1]
    got = np.array([1 if c == "+" else -1 for c in out["S"]], np.int8)
    assert np.array_equal(got, s)


@pytest.mark.gpu
def test_c_program_exchange_labels_stay_a_permutation(program):
    out = _run(program, "labels")
    assert out.startswith("LABELS ok")
    assert int(out.split()[2]) > 0  # some configurations moved
