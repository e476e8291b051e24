"""The oracle's multi-threaded forms (used where the serial oracle would take
minutes: the CPU baseline and the full-length parity runs) equal the serial
oracle: lattices, energy and overlap series, exchange counts and labels bit
for bit; Heisenberg energies up to the order of the FP64 sums."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dim,L,T,threads", [(3, 4, 5, 3), (2, 6, 4, 2), (3, 6, 7, 4)])
def test_omp_pt_run_equals_serial(dim, L, T, threads):
    seed, r, n = 11, 37, 25
    betas = list(1.0 / np.geomspace(0.9, 2.0, T))
    J = oracle.ea_couplings(dim, L, r, seed)
    s0 = np.stack([np.stack([oracle.ising_init(dim, L, seed, oracle.lattice_id(a, r >> 5, t), bit=r & 31)
                             for t in range(T)]) for a in range(2)]).copy()
    a_s, b_s = s0.copy(), s0.copy()
    la = np.tile(np.arange(T, dtype=np.int32), (2, 1))
    lb = la.copy()
    Ea, Qa, acca, pa = oracle.pt_run(dim, L, a_s, betas, seed, r, r >> 5, 3, n, 1, pt_step0=2, J=J, labels=la)
    Eb, Qb, accb, pb = oracle.omp_pt_run(dim, L, b_s, betas, seed, r, r >> 5, 3, n, 1, pt_step0=2, J=J,
                                         labels=lb, threads=threads)
    assert np.array_equal(a_s, b_s)
    assert np.array_equal(Ea, Eb) and np.array_equal(Qa, Qb) and np.array_equal(acca, accb)
    assert np.array_equal(la, lb) and pa == pb
    assert acca.sum() > 0


@pytest.mark.parametrize("dim,L,threads", [(3, 6, 3), (3, 8, 4), (2, 10, 2)])
def test_omp_heis_run_equals_serial(dim, L, threads):
    seed, beta, n = 4, 0.693, 30
    lid = oracle.lattice_id(0, 2, 0)
    a = oracle.heis_init(dim, L, seed, lid)
    b = a.copy()
    Ea, Ma = oracle.heis_run(dim, L, a, beta, seed, lid, 5, n, renorm_every=10)
    Eb, Mb = oracle.omp_heis_run(dim, L, b, beta, seed, lid, 5, n, renorm_every=10, measure_every=3,
                                 threads=threads)
    assert np.array_equal(a, b)
    N = L ** dim
    assert np.allclose(Eb, Ea[2::3], rtol=0, atol=1e-11 * N)
    assert np.allclose(Mb, Ma[2::3], rtol=0, atol=1e-11 * N)
