"""Double-checkerboard multi-hit order (Sec. 3.2, 3.4; cubic tiles in 3D,
Sec. 3.6) on the GPU: shared-memory tile kernels vs the oracle, bit for bit
(lattices and measurement series), across tile sizes, hit counts, both
compound orders and both dimensions."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


def _oracle_run(L, T, k, symmetric, betas, seed, n_compound, dim=2):
    out, E, M = [], [], []
    for t, beta in enumerate(betas):
        lid = oracle.lattice_id(0, 0, t)
        s = oracle.ising_init(dim, L, seed, lid)
        e_t, m_t = [], []
        for m in range(n_compound):
            oracle.dcb_sweeps(L, s, beta, seed, lid, m * k, k, T, k, symmetric, dim=dim)
            e_t.append(oracle.ising_energy(dim, L, s))
            m_t.append(oracle.ising_magnetisation(dim, L, s))
        out.append(s)
        E.append(e_t)
        M.append(m_t)
    return np.stack(out), np.array(E).T, np.array(M).T


@pytest.mark.parametrize("L,T,k,symmetric", [(32, 8, 1, False), (32, 16, 3, True), (64, 16, 2, False),
                                              (96, 16, 4, True), (256, 64, 5, True), (256, 128, 2, False),
                                              (512, 32, 7, True)])
def test_dcb_matches_oracle(L, T, k, symmetric):
    betas, seed, n_compound = [0.3, 0.4407, 0.6], 5, 3
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=3, seed=seed)
    order = B.SPIN_ORDER_DCB_SYMMETRIC if symmetric else B.SPIN_ORDER_DCB
    lat.set_update_order(order, T, k)
    out = lat.run(betas, n_compound * k, measure_every=k)
    s, E, M = _oracle_run(L, T, k, symmetric, betas, seed, n_compound)
    assert np.array_equal(lat.unpack().cpu().numpy()[0, :, 0], s)
    assert np.array_equal(out["E"].view(n_compound, 3).cpu().numpy(), E)
    assert np.array_equal(out["M"].view(n_compound, 3).cpu().numpy(), M)
    assert lat.sweeps_done == n_compound * k


@pytest.mark.parametrize("L,T,k,symmetric", [(16, 8, 1, False), (16, 8, 3, True), (32, 16, 2, False),
                                              (48, 8, 4, True), (64, 16, 3, True), (128, 8, 2, True)])
def test_dcb3_matches_oracle(L, T, k, symmetric):
    """3D, cubic tiles: lattices and E, M after every compound move."""
    betas, seed, n_compound = [0.15, 0.2216544, 0.3], 7, 3
    lat = sp.Lattice(B.SPIN_ISING, 3, L, B.SPIN_I8, n_temps=3, seed=seed)
    order = B.SPIN_ORDER_DCB_SYMMETRIC if symmetric else B.SPIN_ORDER_DCB
    lat.set_update_order(order, T, k)
    out = lat.run(betas, n_compound * k, measure_every=k)
    s, E, M = _oracle_run(L, T, k, symmetric, betas, seed, n_compound, dim=3)
    assert np.array_equal(lat.unpack().cpu().numpy()[0, :, 0], s)
    assert np.array_equal(out["E"].view(n_compound, 3).cpu().numpy(), E)
    assert np.array_equal(out["M"].view(n_compound, 3).cpu().numpy(), M)


def test_dcb3_degenerate_temperatures():
    """beta = 0 (every update flips) and beta = 50 (only dE <= 0 flips)."""
    L, T, k, seed = 16, 8, 3, 13
    lat = sp.Lattice(B.SPIN_ISING, 3, L, B.SPIN_I8, n_temps=2, seed=seed)
    lat.set_update_order(B.SPIN_ORDER_DCB_SYMMETRIC, T, k)
    lat.sweep([0.0, 50.0], 2 * k)
    s, _, _ = _oracle_run(L, T, k, True, [0.0, 50.0], seed, 2, dim=3)
    assert np.array_equal(lat.unpack().cpu().numpy()[0, :, 0], s)


def test_dcb_large_lattice_and_tempering():
    """L = 1024, tile 64, 10 hits, three lattices, then one exchange step
    (orders are orthogonal to the exchange): equal to the oracle."""
    L, T, k, betas, seed = 1024, 64, 10, [0.40, 0.4407, 0.50], 9
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=3, seed=seed)
    lat.set_update_order(B.SPIN_ORDER_DCB_SYMMETRIC, T, k)
    lat.sweep(betas, 2 * k)
    s, _, _ = _oracle_run(L, T, k, True, betas, seed, 2)
    assert np.array_equal(lat.unpack().cpu().numpy()[0, :, 0], s)


def test_dcb_rejects_invalid_settings():
    lat = sp.Lattice(B.SPIN_ISING, 2, 96, B.SPIN_I8, seed=1)
    for tile, hits in ((24, 1), (32, 1), (16, 0), (256, 1)):  # 96/32 = 3 tiles: odd
        with pytest.raises(B.SpinError):
            lat.set_update_order(B.SPIN_ORDER_DCB, tile, hits)
    lat.set_update_order(B.SPIN_ORDER_DCB, 16, 4)
    with pytest.raises(B.SpinError):
        lat.sweep([0.44], 6)  # not whole compound moves
    lat.sweep([0.44], 8)
    lat.set_update_order(B.SPIN_ORDER_CHECKERBOARD)
    lat.sweep([0.44], 3)
    ea = sp.Lattice(B.SPIN_EA, 2, 32, B.SPIN_I8, n_real=2, seed=1)
    with pytest.raises(B.SpinError):
        ea.set_update_order(B.SPIN_ORDER_DCB, 16, 2)
    l3 = sp.Lattice(B.SPIN_ISING, 3, 48, B.SPIN_I8, seed=1)
    for tile in (4, 32, 12):  # 3D takes tiles 8 and 16 only; 48 / 16 = 3 is odd
        with pytest.raises(B.SpinError):
            l3.set_update_order(B.SPIN_ORDER_DCB, tile, 2)
    with pytest.raises(B.SpinError):
        l3.set_update_order(B.SPIN_ORDER_DCB, 16, 2)
