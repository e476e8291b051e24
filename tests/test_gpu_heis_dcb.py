"""The 2D Heisenberg model in the double-checkerboard multi-hit order
(Sec. 4's GPU scheme) against the FP64 oracle: one compound move within
1e-5 away from near-ties, the infinite-temperature equivalence, the
renormalisation rule, a long run in equilibrium, and refused settings."""
import math

import numpy as np
import pytest

import oracle
from tests.stats import binned_mean

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _set(lat, s):
    dev = np.zeros((s.shape[0], 4), np.float32)
    dev[:, :3] = s
    lat.spins.copy_(torch.from_numpy(dev.ravel()))


@pytest.mark.parametrize("T,k,symmetric,variant", [(8, 2, False, 0), (16, 2, True, 2), (32, 1, True, 0)])
def test_one_compound_move_within_tolerance(T, k, symmetric, variant):
    L, seed, beta = 64, 12, 1.1
    lat = sp.Lattice(B.SPIN_HEISENBERG, 2, L, B.SPIN_F32X4, seed=seed)
    lat.set_variant(variant)
    lat.set_update_order(B.SPIN_ORDER_DCB_SYMMETRIC if symmetric else B.SPIN_ORDER_DCB, T, k)
    s0 = oracle.heis_init(2, L, seed, 0).astype(np.float32)
    _set(lat, s0)
    lat.sweep([beta], k)
    got = host(lat.spins).reshape(-1, 4)[:, :3]
    ref = s0.astype(np.float64)
    margin = oracle.heis_dcb_sweeps(2, L, ref, beta, seed, 0, 0, k, T, k, symmetric, want_margin=True)
    err = np.max(np.abs(got - ref), axis=1)
    # a decision taken differently near a tie can spread by one site per
    # fine-colour step: exclude everything within 2 k of a flagged site
    flagged = (margin < 1e-5).reshape(L, L)
    near = flagged.copy()
    for _ in range(2 * k):
        near = near | np.roll(near, 1, 0) | np.roll(near, -1, 0) | np.roll(near, 1, 1) | np.roll(near, -1, 1)
    bad = (err > 1e-5) & ~near.ravel()
    assert not bad.any(), (np.nonzero(bad)[0][:10], err[bad][:10])
    assert near.sum() < L * L // 8


def test_infinite_temperature_keeps_the_last_proposal():
    """At beta = 0 every proposal is accepted: after one compound move the
    lattice equals a plain sweep numbered k - 1 (FP32 vs FP64 unit vectors)."""
    L, T, k, seed = 32, 8, 3, 4
    lat = sp.Lattice(B.SPIN_HEISENBERG, 2, L, B.SPIN_F32X4, seed=seed)
    lat.set_update_order(B.SPIN_ORDER_DCB, T, k)
    lat.sweep([0.0], k)
    got = host(lat.spins).reshape(-1, 4)[:, :3]
    ref = oracle.heis_init(2, L, seed, 0)
    oracle.heis_sweep(2, L, ref, 0.0, seed, 0, k - 1)
    assert np.max(np.abs(got - ref)) < 1e-6


def test_renormalisation_after_moves_passing_100():
    L = 32
    lat = sp.Lattice(B.SPIN_HEISENBERG, 2, L, B.SPIN_F32X4, n_temps=2, seed=6)
    lat.set_update_order(B.SPIN_ORDER_DCB_SYMMETRIC, 16, 40)
    lat.sweep([0.7, 1.4], 120)  # the third move passes 100
    v = host(lat.spins).reshape(-1, 4)[:, :3].astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(v, axis=1) - 1)) <= 1e-6


def test_long_run_energy_matches_fp64_oracle():
    L, beta, T, k, n, seed = 16, 1.1, 8, 2, 2000, 14
    lat = sp.Lattice(B.SPIN_HEISENBERG, 2, L, B.SPIN_F32X4, seed=seed)
    lat.set_update_order(B.SPIN_ORDER_DCB_SYMMETRIC, T, k)
    out = lat.run([beta], n * k, measure_every=k)
    eg = out["Ef"].cpu().numpy() / L ** 2
    s = oracle.heis_init(2, L, seed, 0)
    eo = np.empty(n)
    for m in range(n):
        oracle.heis_dcb_sweeps(2, L, s, beta, seed, 0, m * k, k, T, k, True)
        eo[m] = oracle.heis_energy(2, L, s) / L ** 2
    mg, sg = binned_mean(eg[200:], 30)
    mo, so = binned_mean(eo[200:], 30)
    assert abs(mg - mo) <= 3 * math.sqrt(sg ** 2 + so ** 2) + 1e-12, (mg, sg, mo, so)


def test_refused_settings():
    lat = sp.Lattice(B.SPIN_HEISENBERG, 2, 96, B.SPIN_F32X4, seed=1)
    for tile in (4, 64, 12, 32):  # 96 / 32 = 3 tiles: odd
        with pytest.raises(B.SpinError):
            lat.set_update_order(B.SPIN_ORDER_DCB, tile, 2)
    h3 = sp.Lattice(B.SPIN_HEISENBERG, 3, 16, B.SPIN_F32X4, seed=1)
    with pytest.raises(B.SpinError):
        h3.set_update_order(B.SPIN_ORDER_DCB, 8, 2)
