"""The per-handle autotuner (spin_tune): it picks among the kernel forms of
the int8 ferromagnet, which all give the same chain, and the tile edge of a
double-checkerboard handle left open; the handle's spins and counters are
as before, and the chain continues as on an untuned twin (or one set to the
chosen tile by hand)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


@pytest.mark.parametrize("L,n_real,allowed", [(64, 3, {0, 1, 3}), (512, 2, {0, 1, 4})])
def test_tune_picks_a_variant_and_keeps_the_chain(L, n_real, allowed):
    betas = [0.4407]
    a = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=n_real, seed=12)
    b = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=n_real, seed=12)
    a.sweep(betas, 3)
    b.sweep(betas, 3)
    before = a.spins.clone()
    variant, _ = a.tune(betas, 8)
    assert variant in allowed
    assert torch.equal(a.spins, before) and a.sweeps_done == 3 and a.pt_steps_done == 0
    a.sweep(betas, 8)
    b.sweep(betas, 8)
    assert torch.equal(a.spins, b.spins)
    # every candidate gives that chain
    for v in sorted(allowed):
        c = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=n_real, seed=12)
        c.set_variant(v)
        c.sweep(betas, 11)
        assert torch.equal(c.spins, b.spins), v
        c.close()
    # a handle of the same shape takes the cached choice
    d = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=n_real, seed=3)
    assert d.tune(betas, 8)[0] == variant
    for h in (a, b, d):
        h.close()


@pytest.mark.parametrize("order", [B.SPIN_ORDER_DCB, B.SPIN_ORDER_DCB_SYMMETRIC])
def test_tune_chooses_an_open_tile_edge(order):
    L, k, betas = 256, 4, [0.44, 0.40]
    a = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=2, seed=21)
    a.set_update_order(order, 0, k)
    with pytest.raises(B.SpinError):  # the tile edge is still open
        a.sweep(betas, k)
    before = a.spins.clone()
    _, tile = a.tune(betas, 2 * k)
    assert tile in (8, 16, 32, 64, 128) and L % tile == 0 and (L // tile) % 2 == 0
    assert torch.equal(a.spins, before) and a.sweeps_done == 0
    a.sweep(betas, 2 * k)
    b = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=2, seed=21)
    b.set_update_order(order, tile, k)
    b.sweep(betas, 2 * k)
    assert torch.equal(a.spins, b.spins)
    a.close()
    b.close()


def test_tune_keeps_a_tile_set_by_hand():
    """A handle whose tile edge was chosen by hand keeps it, even after a
    handle of the same shape with an open edge was tuned."""
    L, k, betas = 256, 2, [0.44]
    a = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=5)
    a.set_update_order(B.SPIN_ORDER_DCB, 0, k)
    _, tuned = a.tune(betas, 2 * k)
    fixed = 8 if tuned != 8 else 16
    b = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=5)
    b.set_update_order(B.SPIN_ORDER_DCB, fixed, k)
    assert b.tune(betas, 2 * k)[1] == fixed
    a.close()
    b.close()


def test_tune_rejects_bad_arguments():
    a = sp.Lattice(B.SPIN_ISING, 2, 64, B.SPIN_I8, seed=2)
    with pytest.raises(B.SpinError):
        a.tune([0.44], 0)
    a.set_update_order(B.SPIN_ORDER_DCB, 8, 3)
    with pytest.raises(B.SpinError):  # not a multiple of the hits
        a.tune([0.44], 4)
    a.close()
