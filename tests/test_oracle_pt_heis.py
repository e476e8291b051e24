"""Pins of the oracle's replica exchange (Eq. parallel_tempering) and of its
Heisenberg update (Eq. On_hamiltonian) against exact results."""
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from tests.stats import assert_within, binned_mean


# --------------------------------------------------------------- parallel tempering
def test_pt_slot_marginals_and_swap_rates_match_exact():
    """4x4 ferromagnet (EA lattice with all J = +1), three slots: each slot
    samples its own Boltzmann distribution, and the exchange acceptance of a
    pair equals E[min(1, exp(dbeta dE))] over the product of the two exact
    energy distributions."""
    dim, L = 2, 4
    N = L * L
    betas = np.array([0.3, 0.45, 0.6])
    J = np.ones(dim * N, np.int8)
    spins = np.stack([oracle.ising_init(dim, L, 17, oracle.lattice_id(0, 0, t))
                      for t in range(3)])[None].copy()
    n = 120000
    E, Q, acc, step = oracle.pt_run(dim, L, spins, betas, 17, 0, 0, 0, n, 1, J=J)
    assert step == n
    for t in range(3):
        bf = exact.brute_force(dim, L, betas[t])
        m, err = binned_mean(E[2000:, 0, t])
        assert_within(m, err, bf["E"], what=f"slot {t}")
    for t in range(2):
        l0, p0 = exact.energy_distribution(dim, L, betas[t])
        l1, p1 = exact.energy_distribution(dim, L, betas[t + 1])
        dbeta = betas[t + 1] - betas[t]
        rate = sum(pa * pb * min(1.0, math.exp(dbeta * (eb - ea)))
                   for ea, pa in zip(l0, p0) for eb, pb in zip(l1, p1))
        attempts = n // 2  # pair t is tried on steps with step = t (mod 2)
        got = acc[0, t] / attempts
        assert abs(got - rate) < 0.01, (t, got, rate)
    # the energies carried through the exchanges are those of the configurations
    for t in range(3):
        assert oracle.ising_energy(dim, L, spins[0, t], J) == \
            oracle.ising_energy(dim, L, spins[0, t], None)


def test_pt_step_rules():
    dim, L = 2, 4
    N = L * L
    up = np.ones(N, np.int8)
    chk = np.array([1 if (i % L + i // L) % 2 == 0 else -1 for i in range(N)], np.int8)
    # beta increasing with t: a low-energy configuration held at the smaller
    # beta moves to the larger beta with certainty (Delta > 0)
    E = [oracle.ising_energy(dim, L, up), oracle.ising_energy(dim, L, chk)]
    E2, acc = oracle.pt_step(dim, L, [up.copy(), chk.copy()], E, [0.5, 0.6], 1, 0, 0, 0)
    assert acc[0] == 1 and E2[0] > E2[1]
    # odd step: pair (0, 1) is not tried
    E3, acc = oracle.pt_step(dim, L, [up.copy(), chk.copy()], E, [0.5, 0.6], 1, 0, 0, 1)
    assert acc[0] == 0 and list(E3) == E
    # the reverse exchange against a huge barrier is never accepted
    E4, acc = oracle.pt_step(dim, L, [chk.copy(), up.copy()], E[::-1], [0.5, 5.0], 1, 0, 0, 0)
    assert acc[0] == 0 and list(E4) == E[::-1]


def test_pt_overlap_series():
    dim, L = 3, 4
    N = L ** dim
    betas = [0.9, 1.0]
    J = oracle.ea_couplings(dim, L, 0, seed=4)
    spins = np.stack([np.stack([oracle.ising_init(dim, L, 4, oracle.lattice_id(a, 0, t))
                                for t in range(2)]) for a in range(2)]).copy()
    E, Q, acc, _ = oracle.pt_run(dim, L, spins, betas, 4, 0, 0, 0, 5, 1, J=J)
    for t in range(2):
        assert Q[-1, t] == oracle.overlap(dim, L, spins[0, t], spins[1, t]) or acc.sum() > 0
        assert abs(Q[-1, t]) <= N


# --------------------------------------------------------------- Heisenberg
def test_heis_infinite_temperature_gives_uniform_proposals():
    dim, L = 3, 16
    s = oracle.heis_init(dim, L, 3, 0)
    oracle.heis_sweep(dim, L, s, 0.0, 3, 0, 0)
    norms = np.linalg.norm(s, axis=1)
    assert np.max(np.abs(norms - 1)) < 1e-14
    N = s.shape[0]
    sd = 1 / math.sqrt(N)
    for k in range(3):
        assert abs(s[:, k].mean()) < 5 * sd * math.sqrt(1 / 3)
        assert abs((s[:, k] ** 2).mean() - 1 / 3) < 5 * sd * math.sqrt(4 / 45)
    # z uniform on [-1, 1] (Archimedes): compare quartiles
    q = np.quantile(s[:, 2], [0.25, 0.5, 0.75])
    assert np.max(np.abs(q - np.array([-0.5, 0.0, 0.5]))) < 0.03


def test_heis_chain_correlation_matches_langevin():
    """1D periodic chain: <s_i . s_{i+1}> = coth(beta) - 1/beta exactly."""
    dim, L, beta = 1, 64, 1.5
    s = oracle.heis_init(dim, L, 8, 0)
    E, _ = oracle.heis_run(dim, L, s, beta, 8, 0, 0, 40000)
    m, err = binned_mean(-E[2000:] / L)
    assert_within(m, err, exact.heis_chain_nn(beta, L), what="chain nn")


@pytest.mark.parametrize("dim,L", [(3, 8), (2, 24)])
def test_heis_3d_high_temperature_energy(dim, L):
    """Square and cubic lattices at small beta: the bond correlation is the
    two-spin value coth(beta) - 1/beta up to plaquette corrections of order
    4 u^3 ~ 2e-5."""
    beta = 0.05
    s = oracle.heis_init(dim, L, 2, 0)
    E, _ = oracle.heis_run(dim, L, s, beta, 2, 0, 0, 4000)
    m, err = binned_mean(-E[200:] / (dim * L ** dim))
    assert_within(m, err, exact.langevin(beta), floor=3e-5, what=f"{dim}D bond")


def test_heis_renormalisation_and_energy_definition():
    dim, L = 3, 4
    s = oracle.heis_init(dim, L, 1, 0) * 1.5
    oracle.heis_renormalise(dim, L, s)
    assert np.max(np.abs(np.linalg.norm(s, axis=1) - 1)) < 1e-15
    up = np.zeros((L ** dim, 3))
    up[:, 2] = 1.0
    assert oracle.heis_energy(dim, L, up) == -3 * L ** dim
    assert np.allclose(oracle.heis_magnetisation(dim, L, up), [0, 0, L ** dim])


def test_heis_margins_identify_decisions():
    dim, L, beta = 3, 8, 0.693
    s = oracle.heis_init(dim, L, 4, 0)
    m = oracle.heis_sweep(dim, L, s, beta, 4, 0, 0, want_margin=True)
    assert np.all(m >= 0) and np.all(np.isfinite(m))
