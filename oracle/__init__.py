"""CPU oracle for the checkerboard Metropolis sweep, measurements and replica
exchange of Weigel, arXiv:1101.1427 -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a ctypes wrapper around the
plain serial C in ``spin_oracle.c`` (one int8 per Ising spin, doubles for
Heisenberg spins) plus the closed forms in ``exact.py``; it shares no code
with the CUDA library.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

TAG_UPDATE, TAG_INIT, TAG_COUPLING, TAG_PT, TAG_HEIS, TAG_HEIS_INIT = range(6)


def lib():
    global _lib
    if _lib is None:
        # SPIN_ORACLE_LIB lets the mutation tests load a deliberately broken copy
        path = os.environ.get("SPIN_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        u32, u64, i32, i64, dbl = C.c_uint32, C.c_uint64, C.c_int, C.c_int64, C.c_double
        p = C.c_void_p
        L.or_philox4x32_10.argtypes = [p, p, p]
        L.or_draw.argtypes = [u64, u32, u32, u32, u32, u32, u32]
        L.or_draw.restype = u32
        L.or_lattice_id.argtypes = [u32, u32, u32]
        L.or_lattice_id.restype = u32
        L.or_metropolis_threshold.argtypes = [dbl, i32]
        L.or_metropolis_threshold.restype = u32
        L.or_pt_threshold.argtypes = [dbl, i64]
        L.or_pt_threshold.restype = u32
        L.or_colour.argtypes = [i32, i32, i64]
        L.or_colour.restype = i32
        L.or_ising_init.argtypes = [i32, i32, p, u64, u32, i32, i32]
        L.or_ea_couplings.argtypes = [i32, i32, i32, p, u64]
        L.or_ising_sweep.argtypes = [i32, i32, p, p, dbl, u64, u32, u32, p]
        L.or_ising_energy.argtypes = [i32, i32, p, p]
        L.or_ising_energy.restype = i64
        L.or_ising_magnetisation.argtypes = [i32, i32, p]
        L.or_ising_magnetisation.restype = i64
        L.or_overlap.argtypes = [i32, i32, p, p]
        L.or_overlap.restype = i64
        L.or_pt_step.argtypes = [i32, i32, i32, p, p, p, u64, u32, u32, u32, p, p]
        L.or_heis_init.argtypes = [i32, i32, p, u64, u32]
        L.or_heis_sweep.argtypes = [i32, i32, p, dbl, u64, u32, u32, p]
        L.or_heis_renormalise.argtypes = [i32, i32, p]
        L.or_heis_energy.argtypes = [i32, i32, p]
        L.or_heis_energy.restype = dbl
        L.or_heis_magnetisation.argtypes = [i32, i32, p, p]
        L.or_ising_run.argtypes = [i32, i32, p, p, dbl, u64, u32, u32, i64, p, p, p]
        L.or_heis_run.argtypes = [i32, i32, p, dbl, u64, u32, u32, i64, i32, p, p]
        L.or_pt_run.argtypes = [i32, i32, i32, i32, p, p, p, u64, u32, u32, u32, i64, i32,
                                p, p, p, p, p]
        L.or_ising_window_sweeps.argtypes = [i32, i32, p, i32, p, dbl, u64, u32, u32, i32]
        L.or_ising_init_sites.argtypes = [i64, p, p, u64, u32, i32]
        L.or_dcb_sweeps.argtypes = [i32, p, p, dbl, u64, u32, u32, i64, i32, i32, i32, p]
        L.or_dcb_sweeps_dim.argtypes = [i32, i32, p, p, dbl, u64, u32, u32, i64, i32, i32, i32, p]
        L.or_heis_dcb_sweeps.argtypes = [i32, i32, p, dbl, u64, u32, u32, i64, i32, i32, i32, i32, p]
        L.or_ising_slab_phase.argtypes = [i32, i32, i32, p, dbl, u64, u32, u32, i32, p]
        _lib = L
    return _lib


_omp = None


def omp_lib():
    """The all-cores sweep of the CPU baseline (spin_oracle_omp.c)."""
    global _omp
    if _omp is None:
        L = C.CDLL(_build.build_omp())
        L.or_omp_ising2d_sweeps.argtypes = [C.c_int, C.c_void_p, C.c_double, C.c_uint64, C.c_uint32,
                                            C.c_uint32, C.c_int64, C.c_int, C.c_void_p]
        L.or_omp_ising2d_sweeps.restype = C.c_int64
        p, i32, u32, u64, i64, dbl = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_int64, C.c_double
        L.or_omp_pt_run.argtypes = [i32, i32, i32, i32, p, p, p, u64, u32, u32, u32, i64, i32,
                                    p, p, p, p, p, i32]
        L.or_omp_heis_run.argtypes = [i32, i32, p, dbl, u64, u32, u32, i64, i32, i32, p, p, i32]
        _omp = L
    return _omp


def omp_ising2d_sweeps(L, s, beta, seed, lid, first_sweep, n_sweeps, threads=0):
    """n_sweeps checkerboard sweeps of a 2D L x L int8 ferromagnet in place on
    `threads` host cores (0: all); returns (flips, threads used)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous and s.size == L * L
    used = C.c_int(0)
    f = omp_lib().or_omp_ising2d_sweeps(L, s.ctypes.data_as(C.c_void_p), beta, seed, lid, first_sweep,
                                        n_sweeps, threads, C.byref(used))
    return int(f), used.value


def omp_pt_run(dim, L, spins, betas, seed, r, rkey, first_sweep, n_sweeps, pt_every, pt_step0=0, J=None,
               labels=None, threads=0):
    """pt_run with the lattices of each sweep shared among host threads (the
    same results bit for bit)."""
    n_sets, n_temps, _ = spins.shape
    assert spins.flags.c_contiguous and spins.dtype == np.int8 and n_temps <= 4096 and n_sets <= 2
    b = np.ascontiguousarray(betas, dtype=np.float64)
    E = np.zeros((n_sweeps, n_sets, n_temps), np.int64)
    Q = np.zeros((n_sweeps, n_temps), np.int64)
    acc = np.zeros((n_sets, n_temps), np.int64)
    step = np.array([pt_step0], np.uint32)
    omp_lib().or_omp_pt_run(dim, L, n_temps, n_sets, _ptr(spins), _ptr(J), _ptr(b), seed, r, rkey,
                            first_sweep, n_sweeps, pt_every, _ptr(step), _ptr(E), _ptr(Q), _ptr(acc),
                            _ptr(labels), threads)
    return E, Q, acc, int(step[0])


def omp_heis_run(dim, L, s, beta, seed, lid, first_sweep, n_sweeps, renorm_every=100, measure_every=1,
                 threads=0):
    """heis_run with the sites of each colour phase shared among host threads
    (the lattice equals the serial run bit for bit; E and M are summed in a
    thread-dependent order); measurements after every measure_every sweeps."""
    rows = n_sweeps // measure_every if measure_every > 0 else 0
    E = np.zeros(rows, np.float64)
    M = np.zeros((rows, 3), np.float64)
    omp_lib().or_omp_heis_run(dim, L, _ptr(s), beta, seed, lid, first_sweep, n_sweeps, renorm_every,
                              measure_every, _ptr(E), _ptr(M), threads)
    return E, M


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- RNG
def philox(ctr, key):
    """Philox4x32-10 of a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed, tag, colour, extra, lattice_id, sweep, idx):
    return int(lib().or_draw(seed, tag, colour, extra, lattice_id, sweep, idx))


def lattice_id(a, rkey, t):
    return int(lib().or_lattice_id(a, rkey, t))


def metropolis_threshold(beta, dE):
    return int(lib().or_metropolis_threshold(beta, dE))


def pt_threshold(abs_dbeta, m):
    return int(lib().or_pt_threshold(abs_dbeta, m))


# ---------------------------------------------------------------- Ising / EA
def nsites(dim, L):
    return L ** dim


def ising_init(dim, L, seed, lid, bit=0, hot=True):
    s = np.empty(nsites(dim, L), np.int8)
    lib().or_ising_init(dim, L, _ptr(s), seed, lid, bit, int(hot))
    return s


def ea_couplings(dim, L, r, seed):
    J = np.empty(dim * nsites(dim, L), np.int8)
    lib().or_ea_couplings(dim, L, r, _ptr(J), seed)
    return J


def ising_sweep(dim, L, s, beta, seed, lid, sweep, J=None):
    flips = np.zeros(1, np.int64)
    lib().or_ising_sweep(dim, L, _ptr(s), _ptr(J), beta, seed, lid, sweep, _ptr(flips))
    return int(flips[0])


def ising_energy(dim, L, s, J=None):
    return int(lib().or_ising_energy(dim, L, _ptr(s), _ptr(J)))


def ising_magnetisation(dim, L, s):
    return int(lib().or_ising_magnetisation(dim, L, _ptr(s)))


def overlap(dim, L, s0, s1):
    return int(lib().or_overlap(dim, L, _ptr(s0), _ptr(s1)))


def ising_run(dim, L, s, beta, seed, lid, first_sweep, n_sweeps, J=None, series=True):
    """n_sweeps sweeps in place; returns (E[k], M[k], flips) after each sweep."""
    E = np.zeros(n_sweeps, np.int64) if series else None
    M = np.zeros(n_sweeps, np.int64) if series else None
    flips = np.zeros(1, np.int64)
    lib().or_ising_run(dim, L, _ptr(s), _ptr(J), beta, seed, lid, first_sweep, n_sweeps,
                       _ptr(E), _ptr(M), _ptr(flips))
    return E, M, int(flips[0])


def pt_step(dim, L, slots, E, betas, seed, set_a, r, step, labels=None):
    """One exchange step on a list of per-slot int8 arrays (modified in place);
    labels (int32 [n_temps], optional) are exchanged with the configurations."""
    n_temps = len(slots)
    arr = (C.c_void_p * n_temps)(*[s.ctypes.data for s in slots])
    Ea = np.ascontiguousarray(E, dtype=np.int64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    acc = np.zeros(n_temps, np.int64)
    if labels is not None:
        assert labels.dtype == np.int32 and labels.flags.c_contiguous and labels.size == n_temps
    lib().or_pt_step(dim, L, n_temps, C.cast(arr, C.c_void_p), _ptr(Ea), _ptr(b), seed,
                     set_a, r, step, _ptr(acc), _ptr(labels))
    return Ea, acc


def pt_run(dim, L, spins, betas, seed, r, rkey, first_sweep, n_sweeps, pt_every,
           pt_step0=0, J=None, labels=None):
    """Parallel-tempering run of one realisation; spins [n_sets, n_temps, N]
    int8 (modified in place); labels (int32 [n_sets, n_temps], optional,
    modified in place) follow the configurations through the exchanges.
    Returns (E_series, Q_series, accepted, pt_step)."""
    n_sets, n_temps, _ = spins.shape
    assert spins.flags.c_contiguous and spins.dtype == np.int8
    if labels is not None:
        assert labels.dtype == np.int32 and labels.flags.c_contiguous and labels.shape == (n_sets, n_temps)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    E = np.zeros((n_sweeps, n_sets, n_temps), np.int64)
    Q = np.zeros((n_sweeps, n_temps), np.int64)
    acc = np.zeros((n_sets, n_temps), np.int64)
    step = np.array([pt_step0], np.uint32)
    lib().or_pt_run(dim, L, n_temps, n_sets, _ptr(spins), _ptr(J), _ptr(b), seed, r, rkey,
                    first_sweep, n_sweeps, pt_every, _ptr(step), _ptr(E), _ptr(Q), _ptr(acc),
                    _ptr(labels))
    return E, Q, acc, int(step[0])


def dcb_sweeps(L, s, beta, seed, lid, first_sweep, n_sweeps, T, k, symmetric=False, J=None, dim=2):
    """Double checkerboard multi-hit sweeps of a 2D or 3D int8 lattice in
    place (n_sweeps updates per site, a multiple of k); returns the flip
    count."""
    flips = np.zeros(1, np.int64)
    if dim == 2:
        lib().or_dcb_sweeps(L, _ptr(s), _ptr(J), beta, seed, lid, first_sweep, n_sweeps, T, k,
                            int(bool(symmetric)), _ptr(flips))
    else:
        lib().or_dcb_sweeps_dim(dim, L, _ptr(s), _ptr(J), beta, seed, lid, first_sweep, n_sweeps, T, k,
                                int(bool(symmetric)), _ptr(flips))
    return int(flips[0])


def slab_phase(L, y0, rows, slab, beta, seed, lid, sweep, colour):
    """One colour phase of the own rows of a slab ([rows + 2][L] int8, ghost
    rows 0 and rows + 1) in place; returns the flip count."""
    flips = np.zeros(1, np.int64)
    lib().or_ising_slab_phase(L, y0, rows, _ptr(slab), beta, seed, lid, sweep, colour, _ptr(flips))
    return int(flips[0])


def window_sweeps(dim, L, origin, W, win, beta, seed, lid, first_sweep, n_sweeps):
    o = np.zeros(3, np.int32)
    o[:len(origin)] = origin
    lib().or_ising_window_sweeps(dim, L, _ptr(o), W, _ptr(win), beta, seed, lid,
                                 first_sweep, n_sweeps)


def init_sites(idx, seed, lid, bit=0):
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size, np.int8)
    lib().or_ising_init_sites(idx.size, _ptr(idx), _ptr(out), seed, lid, bit)
    return out


# ---------------------------------------------------------------- Heisenberg
def heis_init(dim, L, seed, lid):
    s = np.empty((nsites(dim, L), 3), np.float64)
    lib().or_heis_init(dim, L, _ptr(s), seed, lid)
    return s


def heis_sweep(dim, L, s, beta, seed, lid, sweep, want_margin=False):
    margin = np.empty(nsites(dim, L), np.float64) if want_margin else None
    lib().or_heis_sweep(dim, L, _ptr(s), beta, seed, lid, sweep, _ptr(margin))
    return margin


def heis_dcb_sweeps(dim, L, s, beta, seed, lid, first_sweep, n_sweeps, T, k, symmetric=False,
                    renorm_every=100, want_margin=False):
    """Heisenberg sweeps in the double-checkerboard multi-hit order, in place;
    returns the per-site smallest decision margin if asked."""
    margin = np.empty(nsites(dim, L), np.float64) if want_margin else None
    lib().or_heis_dcb_sweeps(dim, L, _ptr(s), beta, seed, lid, first_sweep, n_sweeps, T, k,
                             int(bool(symmetric)), renorm_every, _ptr(margin))
    return margin


def heis_renormalise(dim, L, s):
    lib().or_heis_renormalise(dim, L, _ptr(s))


def heis_energy(dim, L, s):
    return float(lib().or_heis_energy(dim, L, _ptr(s)))


def heis_magnetisation(dim, L, s):
    m = np.zeros(3, np.float64)
    lib().or_heis_magnetisation(dim, L, _ptr(s), _ptr(m))
    return m


def heis_run(dim, L, s, beta, seed, lid, first_sweep, n_sweeps, renorm_every=100):
    E = np.zeros(n_sweeps, np.float64)
    M = np.zeros((n_sweeps, 3), np.float64)
    lib().or_heis_run(dim, L, _ptr(s), beta, seed, lid, first_sweep, n_sweeps,
                      renorm_every, _ptr(E), _ptr(M))
    return E, M
