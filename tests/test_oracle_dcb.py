"""Pins of the oracle's double-checkerboard multi-hit order (Sec. 3.2, 3.4):
the exact distribution of the state after one compound move (propagated
over all 2^16 states of a 4 x 4 torus, one single-site Metropolis kernel at
a time in the order the paper describes), the beta = 0 limit, and long-run
sampling against exact enumeration."""
import numpy as np
import pytest

import oracle
from oracle import exact
from tests.stats import assert_within, binned_mean, tau_int

L4, T2 = 4, 2


def _sites(L, T, coarse, colour):
    out = []
    for i in range(L * L):
        x, y = i % L, i // L
        if ((x // T + y // T) & 1) == coarse and ((x + y) & 1) == colour:
            out.append(i)
    return out


def _exact_after_compound(s0, beta, T, k, first_coarse):
    """Distribution over the 2^(L^2) states (bit i set: s_i = -1) after one
    compound move from s0: the tiles of coarse colour `first_coarse` get k
    hits (fine colour 0 sites, then fine colour 1), then the other tiles."""
    L = int(round(np.sqrt(s0.size)))
    n = L * L
    states = np.arange(1 << n, dtype=np.int64)
    spins = 1 - 2 * ((states[:, None] >> np.arange(n)) & 1)  # [state, site]
    nb = []
    for i in range(n):
        x, y = i % L, i // L
        nb.append([((x + 1) % L) + L * y, ((x - 1) % L) + L * y, x + L * ((y + 1) % L), x + L * ((y - 1) % L)])
    dist = np.zeros(1 << n)
    start = int(sum(1 << i for i in range(n) if s0[i] < 0))
    dist[start] = 1.0

    def apply_site(d, i):
        h = spins[:, nb[i]].sum(axis=1)
        dE = 2 * spins[:, i] * h
        p = np.where(dE <= 0, 1.0, np.exp(-beta * dE.astype(np.float64)))
        moved = d * p
        return d * (1.0 - p) + moved[states ^ (1 << i)]

    for cc in range(2):
        coarse = first_coarse ^ cc
        for _ in range(k):
            for colour in range(2):
                for i in _sites(L, T, coarse, colour):
                    dist = apply_site(dist, i)
    return dist, spins


@pytest.mark.parametrize("k,symmetric,compound", [(2, False, 0), (2, True, 1), (3, True, 2), (1, False, 5)])
def test_one_compound_matches_exact_distribution(k, symmetric, compound):
    beta = 0.4
    s0 = np.ones(L4 * L4, np.int8)
    s0[[0, 5, 6, 11, 14]] = -1
    first = 1 if (symmetric and compound % 2 == 1) else 0
    dist, spins = _exact_after_compound(s0, beta, T2, k, first)
    p_down = (dist[:, None] * (spins < 0)).sum(axis=0)
    e_states = -(spins * np.roll(spins.reshape(-1, L4, L4), -1, 2).reshape(-1, L4 * L4)).sum(1) - \
        (spins * np.roll(spins.reshape(-1, L4, L4), -1, 1).reshape(-1, L4 * L4)).sum(1)
    n_samp = 30000
    down = np.zeros(L4 * L4)
    e_hist = {}
    for seed in range(1, n_samp + 1):
        s = s0.copy()
        oracle.dcb_sweeps(L4, s, beta, seed, 0, compound * k, k, T2, k, symmetric)
        down += s < 0
        e = oracle.ising_energy(2, L4, s)
        e_hist[e] = e_hist.get(e, 0) + 1
    freq = down / n_samp
    sig = np.sqrt(np.maximum(p_down * (1 - p_down), 1e-4) / n_samp)
    assert np.all(np.abs(freq - p_down) <= 4.5 * sig), (freq, p_down)
    # energy distribution (chi-square over levels with enough weight)
    levels = np.unique(e_states)
    chi2, dof = 0.0, 0
    for lv in levels:
        p = dist[e_states == lv].sum()
        if p * n_samp >= 20:
            chi2 += (e_hist.get(int(lv), 0) - p * n_samp) ** 2 / (p * n_samp)
            dof += 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_infinite_temperature_flips_every_site_k_times(k):
    """At beta = 0 every Metropolis update flips (threshold 2^32 - 1 misses
    only the word 0xFFFFFFFF), so a compound move multiplies s by (-1)^k."""
    L, T = 16, 4
    lid = oracle.lattice_id(0, 0, 0)
    s0 = oracle.ising_init(2, L, 3, lid)
    s = s0.copy()
    flips = oracle.dcb_sweeps(L, s, 0.0, 3, lid, 0, 4 * k, T, k, True)
    assert flips == 4 * k * L * L
    assert np.array_equal(s, s0)  # 4k flips per site
    s = s0.copy()
    oracle.dcb_sweeps(L, s, 0.0, 3, lid, 0, k, T, k, False)
    assert np.array_equal(s, s0 * (-1) ** k)


@pytest.mark.parametrize("k,symmetric", [(3, True), (4, False)])
def test_long_run_matches_enumeration(k, symmetric):
    beta = 0.4
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.ising_init(2, L4, 17, lid)
    n = 40000
    E = np.empty(n)
    for m in range(n):
        oracle.dcb_sweeps(L4, s, beta, 17, lid, m * k, k, T2, k, symmetric)
        E[m] = oracle.ising_energy(2, L4, s)
    bf = exact.brute_force(2, L4, beta)
    assert (n - 200) / 50 > 20 * tau_int(E[200:])  # bins much longer than the autocorrelation time
    e_mc, e_err = binned_mean(E[200:])
    assert_within(e_mc, e_err, bf["E"], what="<E>")


# ------------------------------------------------------------------ 3D (Sec. 3.6: T x T x T tiles)
def _nb3(L):
    n = L ** 3
    out = []
    for i in range(n):
        x, y, z = i % L, (i // L) % L, i // (L * L)
        out.append([((x + 1) % L) + L * y + L * L * z, ((x - 1) % L) + L * y + L * L * z,
                    x + L * ((y + 1) % L) + L * L * z, x + L * ((y - 1) % L) + L * L * z,
                    x + L * y + L * L * ((z + 1) % L), x + L * y + L * L * ((z - 1) % L)])
    return out


def _sites3(L, T, coarse, colour):
    out = []
    for i in range(L ** 3):
        x, y, z = i % L, (i // L) % L, i // (L * L)
        if ((x // T + y // T + z // T) & 1) == coarse and ((x + y + z) & 1) == colour:
            out.append(i)
    return out


@pytest.mark.parametrize("k,symmetric,compound,start", [(2, False, 0, "up"), (2, True, 1, "mixed"),
                                                         (3, True, 2, "up")])
def test_3d_one_compound_matches_exact_distribution(k, symmetric, compound, start):
    """3D L = 2 (8 sites, 256 states; the periodic neighbours in each
    direction coincide, so every site has each neighbour twice) with T = 1:
    one compound move from a fixed start, sampled over 30000 seeds, against
    the exact distribution propagated one single-site Metropolis kernel at a
    time in the order of the compound move.  From the all-up start every
    first update has dE = 12, so all three thresholds matter."""
    L, T, beta = 2, 1, 0.15
    n = L ** 3
    s0 = np.ones(n, np.int8) if start == "up" else np.array([1, -1, -1, 1, 1, 1, -1, 1], np.int8)
    states = np.arange(1 << n, dtype=np.int64)
    spins = 1 - 2 * ((states[:, None] >> np.arange(n)) & 1)
    nb = _nb3(L)
    dist = np.zeros(1 << n)
    dist[int(sum(1 << i for i in range(n) if s0[i] < 0))] = 1.0
    first = 1 if (symmetric and compound % 2 == 1) else 0
    for cc in range(2):
        for _ in range(k):
            for colour in range(2):
                for i in _sites3(L, T, first ^ cc, colour):
                    dE = 2 * spins[:, i] * spins[:, nb[i]].sum(axis=1)
                    p = np.where(dE <= 0, 1.0, np.exp(-beta * dE.astype(np.float64)))
                    moved = dist * p
                    dist = dist * (1.0 - p) + moved[states ^ (1 << i)]
    n_samp = 30000
    hist = np.zeros(1 << n)
    for seed in range(1, n_samp + 1):
        s = s0.copy()
        oracle.dcb_sweeps(L, s, beta, seed, 0, compound * k, k, T, k, symmetric, dim=3)
        hist[int(sum(1 << i for i in range(n) if s[i] < 0))] += 1
    chi2, dof = 0.0, 0
    for st in range(1 << n):
        e = dist[st] * n_samp
        if e >= 20:
            chi2 += (hist[st] - e) ** 2 / e
            dof += 1
    assert dof >= 10
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)
    assert hist[dist * n_samp < 1e-9].sum() == 0  # no state the exact kernel cannot reach


@pytest.mark.parametrize("T,k", [(2, 1), (4, 2), (2, 3)])
def test_3d_infinite_temperature_flips_every_site_k_times(T, k):
    L = 8
    lid = oracle.lattice_id(0, 0, 0)
    s0 = oracle.ising_init(3, L, 5, lid)
    s = s0.copy()
    flips = oracle.dcb_sweeps(L, s, 0.0, 5, lid, 0, 2 * k, T, k, True, dim=3)
    assert flips == 2 * k * L ** 3 and np.array_equal(s, s0)
    s = s0.copy()
    oracle.dcb_sweeps(L, s, 0.0, 5, lid, 0, k, T, k, False, dim=3)
    assert np.array_equal(s, s0 * (-1) ** k)


@pytest.mark.parametrize("T,k,symmetric", [(2, 2, False), (4, 2, True), (2, 3, True)])
def test_3d_zero_temperature_order_matches_numpy(T, k, symmetric):
    """At beta = 50 every threshold is 0, so only dE <= 0 flips and the chain
    is deterministic: it must equal a numpy implementation of the compound
    move (tiles of one coarse colour, k hits of fine colour 0 then 1, then
    the other coarse colour; whole fine-colour steps at once, as their sites
    are not neighbours)."""
    L = 8
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.ising_init(3, L, 9, lid)
    ref = s.reshape(L, L, L).astype(np.int64)  # [z][y][x]
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    coarse_of = ((x // T + y // T + z // T) & 1)
    colour_of = (x + y + z) & 1
    n_moves = 3
    for m in range(n_moves):
        first = 1 if (symmetric and m % 2 == 1) else 0
        for cc in range(2):
            for _ in range(k):
                for colour in range(2):
                    mask = (coarse_of == (first ^ cc)) & (colour_of == colour)
                    h = sum(np.roll(ref, sh, ax) for ax in range(3) for sh in (1, -1))
                    flip = mask & (2 * ref * h <= 0)
                    ref = np.where(flip, -ref, ref)
    oracle.dcb_sweeps(L, s, 50.0, 9, lid, 0, n_moves * k, T, k, symmetric, dim=3)
    assert np.array_equal(s.reshape(L, L, L), ref)


def test_3d_long_run_matches_enumeration():
    """L = 2, T = 1: <E> over a long chain equals exact enumeration."""
    beta, k = 0.3, 2
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.ising_init(3, 2, 23, lid)
    n = 40000
    E = np.empty(n)
    for m in range(n):
        oracle.dcb_sweeps(2, s, beta, 23, lid, m * k, k, 1, k, True, dim=3)
        E[m] = oracle.ising_energy(3, 2, s)
    assert (n - 200) / 50 > 20 * tau_int(E[200:])
    e_mc, e_err = binned_mean(E[200:])
    assert_within(e_mc, e_err, exact.brute_force(3, 2, beta)["E"], what="<E>")


def test_3d_long_run_matches_plain_sweeps():
    """L = 4, T = 2 (eight 2^3 tiles): the double-checkerboard chain and the
    plain red-black chain sample the same <E> (both stationary for the
    Boltzmann distribution)."""
    beta, k, L = 0.2, 2, 4
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.ising_init(3, L, 29, lid)
    n = 30000
    E = np.empty(n)
    for m in range(n):
        oracle.dcb_sweeps(L, s, beta, 29, lid, m * k, k, 2, k, False, dim=3)
        E[m] = oracle.ising_energy(3, L, s)
    s2 = oracle.ising_init(3, L, 31, lid)
    E2, _, _ = oracle.ising_run(3, L, s2, beta, 31, lid, 0, 2 * n)
    a, ea = binned_mean(E[200:])
    b, eb = binned_mean(E2[400:])
    assert abs(a - b) <= 4.5 * np.hypot(ea, eb), (a, ea, b, eb)


# ------------------------------------------------------------------ Heisenberg (Sec. 4)
@pytest.mark.parametrize("dim,L,T,k,symmetric,move", [(2, 16, 4, 3, True, 1), (2, 16, 8, 2, False, 0),
                                                      (3, 8, 2, 2, True, 3)])
def test_heis_dcb_infinite_temperature_keeps_the_last_proposal(dim, L, T, k, symmetric, move):
    """At beta = 0 every proposal is accepted, so after compound move m every
    site holds the proposal of its last hit, whatever the order: the state
    equals one plain sweep with sweep number m k + k - 1 from any start."""
    lid = oracle.lattice_id(0, 0, 0)
    a = oracle.heis_init(dim, L, 4, lid)
    b = oracle.heis_init(dim, L, 5, lid)  # a different start
    oracle.heis_dcb_sweeps(dim, L, a, 0.0, 4, lid, move * k, k, T, k, symmetric, renorm_every=0)
    oracle.heis_sweep(dim, L, b, 0.0, 4, lid, move * k + k - 1)
    assert np.array_equal(a, b)


def test_heis_dcb_long_run_matches_plain_sweeps():
    """2D L = 8 with 4 x 4 tiles and k = 2: the double-checkerboard chain and
    the plain chain sample the same <E> at beta = 1.1."""
    dim, L, beta, k, T = 2, 8, 1.1, 2, 4
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.heis_init(dim, L, 7, lid)
    n = 6000
    E = np.empty(n)
    for m in range(n):
        oracle.heis_dcb_sweeps(dim, L, s, beta, 7, lid, m * k, k, T, k, True)
        E[m] = oracle.heis_energy(dim, L, s)
    s2 = oracle.heis_init(dim, L, 8, lid)
    E2, _ = oracle.heis_run(dim, L, s2, beta, 8, lid, 0, 2 * n)
    a, ea = binned_mean(E[300:] / L ** 2)
    b, eb = binned_mean(E2[600:] / L ** 2)
    assert abs(a - b) <= 4.5 * np.hypot(ea, eb), (a, ea, b, eb)


def test_heis_dcb_renormalises_when_a_move_passes_a_multiple():
    dim, L, k = 2, 8, 3
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.heis_init(dim, L, 9, lid) * 1.25  # off the unit sphere
    oracle.heis_dcb_sweeps(dim, L, s, 0.7, 9, lid, 0, k, 4, k, renorm_every=4)  # counts 1..3: no multiple of 4
    assert np.max(np.abs(np.linalg.norm(s, axis=1) - 1)) > 0.1
    oracle.heis_dcb_sweeps(dim, L, s, 0.7, 9, lid, k, k, 4, k, renorm_every=4)  # counts 4..6 pass 4
    assert np.max(np.abs(np.linalg.norm(s, axis=1) - 1)) < 1e-14
