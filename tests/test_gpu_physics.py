"""Physics-level checks of the GPU chains: the 2D Ising ferromagnet with
replica exchange (the paper's tempering benchmark, Sec. 6) bit-exact with the
oracle, and long runs of the coded 2D sweep reproducing the exact energy and
specific heat of the 1024 x 1024 torus at beta = 0.4 (Tab. rng)."""
import math
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("L,pt_every,me,n", [(16, 1, 1, 12), (32, 3, 1, 12), (6, 1, 1, 12), (16, 5, 3, 23),
                                             (8, 4200, 7, 4500)])
def test_ising2d_parallel_tempering_bit_exact(L, pt_every, me, n):
    """n = 20 replicas at equally spaced beta in [0.1, 0.15] (Sec. 6), int8
    layout, E every `me` sweeps and one exchange per `pt_every`: lattices,
    energies and exchange counts equal the oracle's.  L % 8 == 0 runs the
    resident kernel, which measures itself; its first stretch of 4200 sweeps
    without an exchange takes two launches (at most 4096 sweeps each), the
    measurement rows continuing across them."""
    n_t, seed = 20, 21
    betas = list(np.linspace(0.1, 0.15, n_t))
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=n_t, seed=seed)
    acc = torch.zeros(n_t, dtype=torch.int64, device="cuda")
    labels = lat.slot_labels()
    out = lat.run(betas, n, me, pt_every, accepted=acc, labels=labels)
    s = np.stack([oracle.ising_init(2, L, seed, oracle.lattice_id(0, 0, t)) for t in range(n_t)])[None].copy()
    lab = np.arange(n_t, dtype=np.int32)[None].copy()
    Es, _, acc_o, _ = oracle.pt_run(2, L, s, betas, seed, 0, 0, 0, n, pt_every, labels=lab)
    assert np.array_equal(lat.unpack().cpu().numpy()[:, :, 0], s)
    assert np.array_equal(out["E"].view(n // me, 1, n_t).cpu().numpy(), Es[me - 1::me])
    assert np.array_equal(acc.cpu().numpy(), acc_o[0])
    assert np.array_equal(labels.view(1, n_t).cpu().numpy(), lab)


@pytest.mark.parametrize("L,pt_every,me,n", [(8, 2, 1, 9), (16, 4, 3, 12), (24, 1, 1, 5), (12, 2, 1, 6)])
def test_ising3d_parallel_tempering_bit_exact(L, pt_every, me, n):
    """The 3D ferromagnet with replica exchange: 10 int8 replicas around the
    critical coupling, E every `me` sweeps; L % 8 == 0 (L <= 24) runs the
    resident kernel, which measures itself, L = 12 the colour phases."""
    n_t, seed = 10, 23
    betas = list(np.linspace(0.18, 0.26, n_t))
    lat = sp.Lattice(B.SPIN_ISING, 3, L, B.SPIN_I8, n_temps=n_t, seed=seed)
    acc = torch.zeros(n_t, dtype=torch.int64, device="cuda")
    out = lat.run(betas, n, me, pt_every, accepted=acc)
    s = np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(0, 0, t)) for t in range(n_t)])[None].copy()
    Es, _, acc_o, _ = oracle.pt_run(3, L, s, betas, seed, 0, 0, 0, n, pt_every)
    assert np.array_equal(lat.unpack().cpu().numpy()[:, :, 0], s)
    assert np.array_equal(out["E"].view(n // me, 1, n_t).cpu().numpy(), Es[me - 1::me])
    assert np.array_equal(acc.cpu().numpy(), acc_o[0])
    if n % me == 0 and n % pt_every != 0:  # last row measured after the last exchange
        M = out["M"].view(n // me, n_t).cpu().numpy()[-1]
        assert np.array_equal(M, s[0].astype(np.int64).sum(axis=1))


def _exact_row():
    for line in open(os.path.join(HERE, "golden", "tab_rng_exact.txt")):
        if line.strip() and not line.startswith("#"):
            L, beta, e, cv = line.split()
            return int(L), float(beta), float(e), float(cv)


def test_ising2d_L1024_energy_and_specific_heat_match_exact():
    """Sixteen independent coded L = 1024 chains at beta = 0.4, 50000 sweeps:
    energy per spin and specific heat within 4 standard errors (binned over
    sweeps, then over chains) of the exact torus values."""
    L, beta, e_exact, cv_exact = _exact_row()
    n_chain, n, burn, nbin = 16, 50000, 1000, 49
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=n_chain, seed=31)
    out = lat.run([beta] * n_chain, n, 1)
    E = out["E"].view(n, n_chain).cpu().numpy()[burn:].astype(np.float64)
    N = L * L
    e = -E / N                                   # energy per spin, sign of Tab. rng
    bins = e.reshape(nbin, -1, n_chain)          # [bin][sweep][chain]
    e_bin = bins.mean(axis=1).ravel()
    e_mean = e_bin.mean()
    e_err = e_bin.std(ddof=1) / math.sqrt(e_bin.size)
    assert abs(e_mean - e_exact) <= 4 * e_err, (e_mean, e_err, e_exact)
    # specific heat per spin, beta^2 N var(e), per chain with jackknife over bins
    cv_est = []
    for c in range(n_chain):
        x = bins[:, :, c]
        jk = []
        for k in range(nbin):
            y = np.delete(x, k, axis=0).ravel()
            jk.append(beta * beta * N * y.var())
        jk = np.array(jk)
        full = beta * beta * N * x.ravel().var()
        cv_est.append((full, math.sqrt((nbin - 1) / nbin * ((jk - jk.mean()) ** 2).sum())))
    cv = np.mean([v for v, _ in cv_est])
    cv_err = math.sqrt(sum(s * s for _, s in cv_est)) / n_chain
    assert abs(cv - cv_exact) <= 4 * cv_err, (cv, cv_err, cv_exact)
