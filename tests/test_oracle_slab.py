"""The slab decomposition of a 2D lattice (several GPUs, each owning a band
of rows, exchanging one boundary row with each neighbour before every colour
phase) reproduces the unsplit oracle sweep bit for bit, for any number of
slabs and uneven heights: the random words are keyed by global site index."""
import numpy as np
import pytest

import oracle


def _split(L, P):
    edges = [round(k * L / P) for k in range(P + 1)]
    return [(edges[k], edges[k + 1] - edges[k]) for k in range(P)]


def _slab_sweeps(s_full, L, P, beta, seed, lid, n):
    parts = _split(L, P)
    slabs = []
    for y0, rows in parts:
        sl = np.zeros((rows + 2, L), np.int8)
        sl[1:rows + 1] = s_full.reshape(L, L)[y0:y0 + rows]
        slabs.append(sl)
    for sweep in range(n):
        for colour in (0, 1):
            for k, sl in enumerate(slabs):  # ghost rows from the neighbours (periodic in y)
                above, below = slabs[k - 1], slabs[(k + 1) % P]
                sl[0] = above[-2]
                sl[-1] = below[1]
            for (y0, rows), sl in zip(parts, slabs):
                oracle.slab_phase(L, y0, rows, sl, beta, seed, lid, sweep, colour)
    return np.concatenate([sl[1:-1] for sl in slabs]).ravel()


@pytest.mark.parametrize("L,P", [(16, 1), (16, 2), (24, 3), (30, 4), (32, 5)])
def test_slabs_equal_unsplit_sweeps(L, P):
    beta, seed, n = 0.44, 13, 6
    lid = oracle.lattice_id(0, 0, 0)
    s0 = oracle.ising_init(2, L, seed, lid)
    ref = s0.copy()
    for sweep in range(n):
        oracle.ising_sweep(2, L, ref, beta, seed, lid, sweep)
    got = _slab_sweeps(s0, L, P, beta, seed, lid, n)
    assert np.array_equal(got, ref)
    assert not np.array_equal(ref, s0)


def test_slab_reads_ghosts_only():
    """Changing a ghost row changes the update of the adjacent own row only
    through the field, and the ghost rows themselves are never written."""
    L, rows = 16, 4
    lid = oracle.lattice_id(0, 0, 0)
    sl = np.ones((rows + 2, L), np.int8)
    sl[0] = -1
    before = sl[[0, -1]].copy()
    oracle.slab_phase(L, 3, rows, sl, 0.0, 1, lid, 0, 0)
    assert np.array_equal(sl[[0, -1]], before)
    # at beta = 0 every updated site flips: the colour-0 sites of own rows
    ys = 3 + np.arange(rows)[:, None]
    xs = np.arange(L)[None, :]
    assert np.array_equal(sl[1:-1] == -1, ((xs + ys) & 1) == 0)


@pytest.mark.parametrize("L,threads", [(16, 3), (64, 4), (66, 7)])
def test_openmp_sweep_equals_serial_sweep(L, threads):
    """The all-cores sweep of the CPU baseline (rows of each colour phase
    shared among threads) equals the serial oracle sweep bit for bit."""
    seed, beta, n = 5, 0.4407, 6
    lid = oracle.lattice_id(0, 1, 0)
    s = oracle.ising_init(2, L, seed, lid)
    t = s.copy()
    _, _, flips = oracle.ising_run(2, L, s, beta, seed, lid, 3, n, series=False)
    f2, used = oracle.omp_ising2d_sweeps(L, t, beta, seed, lid, 3, n, threads)
    assert np.array_equal(s, t)
    assert f2 == flips
    assert used >= 1
