"""Pins of the oracle's random numbers and acceptance thresholds.

The Philox4x32-10 of the oracle is checked against cuRAND's host-side
Philox4x32-10 generator (a library call, independent of our code); the
integer thresholds against a 50-digit evaluation of floor(p * 2^32)."""
import ctypes
import os

import mpmath
import numpy as np
import pytest

import oracle


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    cu = _curand()
    if cu is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert cu.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert cu.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 65536 * 3
        out = np.zeros(n, np.uint32)
        assert cu.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        cu.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # cuRAND's host ordering: output 4*(65536*X + s) + w is word w of the
    # block with counter (X, 0, s, 0), the subsequence s in counter word 2.
    rng = np.random.default_rng(7)
    for X in range(3):
        for s in list(range(8)) + list(rng.integers(8, 65536, 40)):
            k = 4 * (65536 * X + int(s))
            assert list(oracle.philox([X, 0, int(s), 0], key)) == list(out[k:k + 4]), (X, s)


def test_draw_uses_counter_layout():
    seed = 99
    key = [seed, 0]
    for idx in (0, 1, 2, 3, 4, 7, 1001):
        ctr = [idx >> 2, 17, 0x01002003, (3 << 28) | (1 << 27) | 5]
        assert oracle.draw(seed, 3, 1, 5, 0x01002003, 17, idx) == oracle.philox(ctr, key)[idx & 3]


def test_lattice_id_packing():
    assert oracle.lattice_id(1, 2, 3) == (1 << 24) | (2 << 12) | 3


def _exact_threshold(p_expr):
    with mpmath.workdps(50):
        t = mpmath.floor(p_expr * mpmath.mpf(2) ** 32)
        return min(int(t), 2 ** 32 - 1)


@pytest.mark.parametrize("beta", [0.0, 0.1, 0.4, 0.4407, 0.5, 0.693, 0.9, 1.1111, 2.0, 10.0])
def test_metropolis_thresholds(beta):
    for dE in (4, 8, 12):
        got = oracle.metropolis_threshold(beta, dE)
        with mpmath.workdps(50):
            x = mpmath.exp(-mpmath.mpf(beta) * dE) * mpmath.mpf(2) ** 32
        exact = min(int(mpmath.floor(x)), 2 ** 32 - 1)
        frac = float(x - mpmath.floor(x))
        if 1e-6 < frac < 1 - 1e-6:  # away from an integer: double must agree
            assert got == exact, (beta, dE)
        else:
            assert abs(got - exact) <= 1
    # infinite temperature: every increase is accepted up to 2^-32
    assert oracle.metropolis_threshold(0.0, 4) == 2 ** 32 - 1


def test_pt_thresholds():
    for dbeta in (0.0, 0.013, 0.02, 0.1, 1.0):
        for m in (0, 1, 5, 50, 300):
            got = oracle.pt_threshold(dbeta, m)
            with mpmath.workdps(50):
                x = mpmath.exp(-mpmath.mpf(dbeta) * 4 * m) * mpmath.mpf(2) ** 32
            exact = min(int(mpmath.floor(x)), 2 ** 32 - 1)
            assert abs(got - exact) <= 1
    assert oracle.pt_threshold(1.0, 10 ** 6) == 0
