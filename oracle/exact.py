"""Closed forms and exhaustive enumerations that pin the CPU oracle
(test infrastructure only).

* ``brute_force``: exact Boltzmann averages of a small Ising / +-J lattice by
  enumerating all 2^N states (the Hamiltonians of Eq. ising_hamiltonian and
  Eq. spinglass_hamiltonian written out as an explicit bond list).
* ``kaufman_torus``: exact partition function of the L x L Ising torus
  (Kaufman 1949, in the form of Ferdinand & Fisher 1969, the reference the
  paper uses for the exact values of Tab. rng), evaluated with mpmath; the
  energy and specific heat are its first and second beta-derivatives.
* ``onsager_energy`` / ``yang_magnetisation``: infinite-lattice closed forms
  (critical coupling beta_c = ln(1 + sqrt 2)/2, Sec. 3.4).
* ``langevin``: <cos theta> of a classical unit vector in a field, the exact
  single-site and 1D-chain nearest-neighbour correlation of the Heisenberg
  model (Eq. On_hamiltonian with n = 3).
"""
import itertools
import math

import mpmath
import numpy as np

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


# ----------------------------------------------------------------- bonds
def bond_list(dim, L, J=None):
    """(i, j, J_ij) for every bond (i, i + e_d), periodic, site index
    i = x + L*y + L*L*z.  J (optional) is laid out [d][site] with +-1."""
    N = L ** dim
    bonds = []
    for site in range(N):
        c = [(site // L ** k) % L for k in range(dim)]
        for d in range(dim):
            c2 = list(c)
            c2[d] = (c2[d] + 1) % L
            nb = sum(c2[k] * L ** k for k in range(dim))
            bonds.append((site, nb, 1 if J is None else int(J[d * N + site])))
    return bonds


def all_states(N):
    """All 2^N spin configurations as an int8 array [2^N, N] of +-1."""
    idx = np.arange(2 ** N, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(N, dtype=np.int64)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def state_energies(dim, L, J=None):
    """Energies of all 2^N states and their magnetisations."""
    N = L ** dim
    S = all_states(N).astype(np.int64)
    E = np.zeros(S.shape[0], np.int64)
    for i, j, jv in bond_list(dim, L, J):
        E -= jv * S[:, i] * S[:, j]
    M = S.sum(axis=1)
    return E, M


def brute_force(dim, L, beta, J=None):
    """Exact <E>, <E^2>, <|M|>, <M^2> at inverse temperature beta."""
    E, M = state_energies(dim, L, J)
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    avg = lambda x: float((w * x).sum() / Z)
    return {"E": avg(E), "E2": avg(E.astype(np.float64) ** 2), "absM": avg(np.abs(M)),
            "M2": avg(M.astype(np.float64) ** 2)}


def energy_distribution(dim, L, beta, J=None):
    """Exact Boltzmann distribution of the energy: (levels, probabilities)."""
    E, _ = state_energies(dim, L, J)
    levels, counts = np.unique(E, return_counts=True)
    logw = np.log(counts) - beta * (levels - levels.min())
    p = np.exp(logw - logw.max())
    return levels, p / p.sum()


# ----------------------------------------------------------------- Kaufman
def _log_kaufman_Z(K, L):
    """ln Z of the L x L periodic Ising model at coupling K = beta J."""
    K = mpmath.mpf(K)
    c = mpmath.cosh(2 * K) * mpmath.coth(2 * K)
    gam = []
    for l in range(2 * L):
        if l == 0:
            gam.append(2 * K + mpmath.log(mpmath.tanh(K)))
        else:
            gam.append(mpmath.acosh(c - mpmath.cos(mpmath.pi * l / L)))
    half = mpmath.mpf(L) / 2
    z1 = z2 = z3 = z4 = mpmath.mpf(1)
    for r in range(L):
        go, ge = gam[2 * r + 1], gam[2 * r]
        z1 *= 2 * mpmath.cosh(half * go)
        z2 *= 2 * mpmath.sinh(half * go)
        z3 *= 2 * mpmath.cosh(half * ge)
        z4 *= 2 * mpmath.sinh(half * ge)
    pref = (mpmath.mpf(L) * L / 2) * mpmath.log(2 * mpmath.sinh(2 * K)) - mpmath.log(2)
    return pref + mpmath.log(z1 + z2 + z3 + z4)


def kaufman_torus(L, beta, dps=40):
    """Exact (e, c_v) of the L x L torus: e = -<E>/N (the sign convention of
    Tab. rng, where e is printed positive) and c_v = beta^2 Var(E)/N."""
    with mpmath.workdps(dps):
        f = lambda b: _log_kaufman_Z(b, L)
        b = mpmath.mpf(beta)
        d1 = mpmath.diff(f, b, 1)
        d2 = mpmath.diff(f, b, 2)
        N = L * L
        return float(d1 / N), float(b * b * d2 / N)


def kaufman_log_Z(L, beta, dps=40):
    with mpmath.workdps(dps):
        return float(_log_kaufman_Z(mpmath.mpf(beta), L))


# ----------------------------------------------------------------- Onsager
def onsager_energy(beta):
    """Infinite-lattice energy per spin u = <E>/N of the square-lattice Ising model."""
    with mpmath.workdps(30):
        K = mpmath.mpf(beta)
        k = 2 * mpmath.sinh(2 * K) / mpmath.cosh(2 * K) ** 2
        K1 = mpmath.ellipk(k * k)
        return float(-mpmath.coth(2 * K) * (1 + 2 / mpmath.pi * (2 * mpmath.tanh(2 * K) ** 2 - 1) * K1))


def yang_magnetisation(beta):
    """Spontaneous magnetisation per spin (0 above T_c)."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2 * beta) ** -4) ** 0.125


# ----------------------------------------------------------------- Heisenberg
def langevin(x):
    """coth(x) - 1/x: <s . e_h> of a unit 3-vector with weight exp(x s . e_h)."""
    if abs(x) < 1e-4:
        return x / 3.0
    return 1.0 / math.tanh(x) - 1.0 / x


def heis_chain_nn(beta, L):
    """Exact nearest-neighbour correlation <s_i . s_{i+1}> of the periodic
    classical Heisenberg chain of L sites: with u = langevin(beta), the
    transfer-operator eigenvalues give (u + u^(L-1)) / (1 + u^L) -- up to
    terms of relative order u^L from higher harmonics, negligible here."""
    u = langevin(beta)
    return (u + u ** (L - 1)) / (1.0 + u ** L)
