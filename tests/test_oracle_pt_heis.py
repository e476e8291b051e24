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


@pytest.mark.parametrize("T", [5, 6])
def test_pt_labels_reverse_after_T_steps_when_every_exchange_is_accepted(T):
    """Equal betas make Delta = 0, so every tried pair is exchanged: the step
    schedule (pairs t = p mod 2) is then the odd-even transposition network,
    which reverses the order of T items in T steps (it sorts a reversed list
    in T rounds, swapping at every comparator) and restores it after 2T."""
    dim, L = 2, 4
    slots = [oracle.ising_init(dim, L, 3, oracle.lattice_id(0, 0, t)) for t in range(T)]
    E = [oracle.ising_energy(dim, L, s) for s in slots]
    labels = np.arange(T, dtype=np.int32)
    for step in range(2 * T):
        E, _ = oracle.pt_step(dim, L, slots, E, [0.7] * T, 3, 0, 0, step, labels=labels)
        if step == T - 1:
            assert list(labels) == list(range(T - 1, -1, -1))
    assert list(labels) == list(range(T))


def test_pt_labels_follow_the_configurations():
    """Distinct configurations at geometric betas, exchange steps without
    sweeps: after every step each slot holds the configuration its label
    names (with that configuration's energy), and the labels stay a
    permutation."""
    dim, L, T = 2, 4, 7
    init = [oracle.ising_init(dim, L, 8, oracle.lattice_id(0, 0, t)) for t in range(T)]
    E0 = [oracle.ising_energy(dim, L, s) for s in init]
    slots = [s.copy() for s in init]
    betas = 0.2 * 1.35 ** np.arange(T)
    E = list(E0)
    labels = np.arange(T, dtype=np.int32)
    moved = 0
    for step in range(400):
        E, acc = oracle.pt_step(dim, L, slots, E, betas, 8, 0, 0, step, labels=labels)
        moved += int(acc.sum())
        assert sorted(labels) == list(range(T))
        for t in range(T):
            assert np.array_equal(slots[t], init[labels[t]])
            assert E[t] == E0[labels[t]]
    assert moved > 50


def test_overlap_definition_cases():
    """q = sum_i s_i^(0) s_i^(1): a configuration with itself gives N, with
    its reversal -N, and q is unchanged when both replicas take the same
    gauge transformation s_i -> eps_i s_i (Eq. spinglass_hamiltonian: the
    transformation that maps one coupling realisation onto another)."""
    dim, L = 3, 6
    N = L ** dim
    s0 = oracle.ising_init(dim, L, 5, oracle.lattice_id(0, 0, 0))
    s1 = oracle.ising_init(dim, L, 5, oracle.lattice_id(1, 0, 0))
    assert oracle.overlap(dim, L, s0, s0) == N
    assert oracle.overlap(dim, L, s0, (-s0).astype(np.int8)) == -N
    eps = oracle.ising_init(dim, L, 6, oracle.lattice_id(0, 7, 0))
    q = oracle.overlap(dim, L, s0, s1)
    assert oracle.overlap(dim, L, (eps * s0).astype(np.int8), (eps * s1).astype(np.int8)) == q
    # sites where the replicas agree minus sites where they differ
    assert q == N - 2 * int(np.count_nonzero(s0 != s1))


def test_overlap_of_independent_replicas_at_infinite_temperature():
    """beta = 0: independent hot starts give <q> = 0 and <q^2> = N (q is a
    sum of N independent +-1 products), and since every site then flips in
    every sweep, the overlap series of a two-set run is constant in time."""
    dim, L = 3, 4
    N = L ** dim
    qs = np.array([oracle.overlap(dim, L, oracle.ising_init(dim, L, 9, oracle.lattice_id(0, k, 0)),
                                  oracle.ising_init(dim, L, 9, oracle.lattice_id(1, k, 0)))
                   for k in range(4000)], np.float64)
    assert abs(qs.mean()) < 4 * np.sqrt(N / qs.size)
    # Var(q^2) = 2 N^2 - 2 N for a sum of N independent signs
    assert abs((qs ** 2).mean() - N) < 4 * np.sqrt((2 * N * N - 2 * N) / qs.size)
    J = oracle.ea_couplings(dim, L, 3, seed=9)
    spins = np.stack([oracle.ising_init(dim, L, 9, oracle.lattice_id(a, 0, 0), bit=3)[None]
                      for a in range(2)]).copy()
    q0 = oracle.overlap(dim, L, spins[0, 0], spins[1, 0])
    _, Q, _, _ = oracle.pt_run(dim, L, spins, [0.0], 9, 3, 0, 0, 6, 0, J=J)
    assert np.all(Q[:, 0] == q0)


def test_overlap_second_moment_matches_enumeration():
    """Two independent replicas of one 4x4 +-J realisation (Sec. 5): the
    overlap series of the oracle's two-set run has <q> = 0 (each replica is
    spin-flip symmetric) and <q^2> = sum_ij <s_i s_j>^2, the correlation
    matrix taken over all 2^16 states."""
    dim, L, beta = 2, 4, 0.6
    N = L * L
    J = oracle.ea_couplings(dim, L, 1, seed=12)
    E_all, _ = exact.state_energies(dim, L, J)
    S = exact.all_states(N).astype(np.float64)
    w = np.exp(-beta * (E_all - E_all.min()))
    p = w / w.sum()
    C = S.T @ (S * p[:, None])
    q2_exact = float((C ** 2).sum())
    spins = np.stack([oracle.ising_init(dim, L, 12, oracle.lattice_id(a, 0, 0), bit=1)[None]
                      for a in range(2)]).copy()
    n = 150000
    _, Q, _, _ = oracle.pt_run(dim, L, spins, [beta], 12, 1, 0, 0, n, 0, J=J)
    q = Q[1000:, 0].astype(np.float64)
    m, err = binned_mean(q)
    assert_within(m, err, 0.0, what="<q>")
    m2, err2 = binned_mean(q ** 2)
    assert_within(m2, err2, q2_exact, what="<q^2>")
    assert N < q2_exact < N * N


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


@pytest.mark.parametrize("beta", [0.0, 0.05])
def test_heis_magnetisation_second_moment(beta):
    """<|M|^2> / N = sum_j <s_0 . s_j>: at beta = 0 every proposal is
    accepted, so each sweep leaves N fresh independent unit vectors and the
    value is exactly 1 (1/3 per component); at small beta the
    high-temperature series of the classical Heisenberg model on the simple
    cubic lattice (6 neighbours; no closed loop below four bonds) gives
    1 + 6u + 30u^2 + 150u^3 + O(u^4), u = coth(beta) - 1/beta."""
    dim, L, n = 3, 8, 20000
    N = L ** dim
    s = oracle.heis_init(dim, L, 21, 0)
    _, M = oracle.heis_run(dim, L, s, beta, 21, 0, 0, n)
    u = exact.langevin(beta)
    chi = 1 + 6 * u + 30 * u * u + 150 * u ** 3
    m2, err = binned_mean((M[100:] ** 2).sum(axis=1) / N)
    assert_within(m2, err, chi, floor=1e-4, what="<|M|^2>/N")
    for k in range(3):
        mk, ek = binned_mean(M[100:, k] ** 2 / N)
        assert_within(mk, ek, chi / 3, floor=1e-4, what=f"<M_{k}^2>/N")
        m1, e1 = binned_mean(M[100:, k] / N)
        assert_within(m1, e1, 0.0, what=f"<M_{k}>/N")


def test_heis_margins_identify_decisions():
    dim, L, beta = 3, 8, 0.693
    s = oracle.heis_init(dim, L, 4, 0)
    m = oracle.heis_sweep(dim, L, s, beta, 4, 0, 0, want_margin=True)
    assert np.all(m >= 0) and np.all(np.isfinite(m))
