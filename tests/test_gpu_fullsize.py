"""Parity at the full sizes of the hot-path configurations, in the launch
forms the benchmark times: sampled outputs that the oracle computes one by
one (light-cone windows, single realisations) or properties that hold at any
size."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402
from tests.stats import binned_mean  # noqa: E402


def _windows(L, rng, count, W):
    origins = [(L - W // 2, L - W // 2), (0, 0), (L - W, 7)]  # wrap-around corners
    origins += [tuple(int(v) for v in rng.integers(0, L, 2)) for _ in range(count - len(origins))]
    return origins


@pytest.mark.parametrize("layout", [B.SPIN_I8, B.SPIN_MSC1])
def test_ising2d_L16384_sampled_windows(layout):
    """2D Ising L=16384, three betas, two sweeps, in the benchmark's layouts:
    every sampled window's interior equals the oracle's light-cone sweeps."""
    L, seed, betas, n, W = 16384, 1, [0.40, 0.4407, 0.50], 2, 14
    lat = sp.Lattice(B.SPIN_ISING, 2, L, layout, n_temps=3, seed=seed)
    lat.sweep(betas, n)
    full = lat.unpack().view(3, L, L)
    rng = np.random.default_rng(5)
    for t, beta in enumerate(betas):
        lid = oracle.lattice_id(0, 0, t)
        for (ox, oy) in _windows(L, rng, 5, W):
            gx = (ox + np.arange(W)) % L
            gy = (oy + np.arange(W)) % L
            idx = (gy[:, None] * L + gx[None, :]).ravel()
            win = oracle.init_sites(idx, seed, lid)
            oracle.window_sweeps(2, L, (ox, oy), W, win, beta, seed, lid, 0, n)
            got = full[t][torch.as_tensor(gy, device="cuda")][:, torch.as_tensor(gx, device="cuda")]
            got = got.cpu().numpy()
            inner = slice(2 * n, W - 2 * n)
            assert np.array_equal(got[inner, inner], win.reshape(W, W)[inner, inner]), (t, ox, oy)


def test_ising2d_L16384_energy_consistent_with_state():
    """The reductions the benchmark times agree with an independent count on
    the unpacked state (a property at any size)."""
    L = 16384
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=3, seed=4)
    lat.sweep([0.40, 0.4407, 0.50], 3)
    E, M, _ = lat.measure()
    s = lat.unpack().view(3, L, L).to(torch.int32)
    E2 = -(s * torch.roll(s, -1, 2)).sum((1, 2)) - (s * torch.roll(s, -1, 1)).sum((1, 2))
    assert torch.equal(E, E2.to(torch.int64)) and torch.equal(M, s.sum((1, 2)).to(torch.int64))


def test_ising3d_L128_full_lattice():
    """3D Ising ferromagnet L = 128 (2^21 int8 sites) at the critical
    coupling, three sweeps by the 3D chunk kernel: the whole lattice equals
    the oracle, and E, M agree with the state."""
    L, seed, beta, n = 128, 17, 0.2216, 3
    lat = sp.Lattice(B.SPIN_ISING, 3, L, B.SPIN_I8, seed=seed)
    lat.sweep([beta], n)
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.ising_init(3, L, seed, lid)
    oracle.ising_run(3, L, s, beta, seed, lid, 0, n, series=False)
    assert np.array_equal(lat.spins.cpu().numpy(), s)
    E, M, _ = lat.measure()
    v = lat.spins.view(L, L, L).to(torch.int32)
    E2 = -sum((v * torch.roll(v, -1, d)).sum() for d in range(3))
    assert int(E[0]) == int(E2) and int(M[0]) == int(v.sum())


def test_ea_L16_full_size_batched_sampled_realisations():
    """3D EA L=16, 1024 realisations x 32 slots x 2 sets, exchange and
    measurement every sweep, in the batched persistent launch: sampled
    realisations equal the oracle run of that realisation alone."""
    L, seed, n = 16, 3, 6
    betas = list(1.0 / np.geomspace(0.9, 2.0, 32))
    lat = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=1024, n_temps=32, n_sets=2, seed=seed)
    ser = lat.series_buffers(n)
    acc = torch.zeros(64, dtype=torch.int64, device="cuda")
    sp.batch_run([lat.batch_item(betas, ser, acc)], n, 1, 1)
    lat.sync()
    got = lat.unpack()
    E = ser["E"].view(n, 2, 32, 1024)
    Q = ser["Q"].view(n, 32, 1024)
    for r in (0, 517, 1023):
        J = oracle.ea_couplings(3, L, r, seed)
        s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(a, r >> 5, t), bit=r & 31)
                                for t in range(32)]) for a in range(2)]).copy()
        Es, Qs, _, _ = oracle.pt_run(3, L, s, betas, seed, r, r >> 5, 0, n, 1, J=J)
        assert np.array_equal(got[:, :, r].cpu().numpy(), s), r
        assert np.array_equal(E[:, :, :, r].cpu().numpy(), Es), r
        assert np.array_equal(Q[:, :, r].cpu().numpy(), Qs), r


def test_ea_L16_full_size_long_run_first_and_last_group():
    """3D EA L=16, 1024 realisations x 32 slots x 2 sets, exchange and
    measurement every sweep for the configuration's full 10^4 sweeps in one
    batched launch: one realisation of the first and one of the last group
    of 32 equal their oracle runs (lattices, energy and overlap series every
    sweep, exchange counts and configuration labels), the oracle running on
    the host cores while the GPU works."""
    from concurrent.futures import ThreadPoolExecutor
    L, seed, n = 16, 9, 10000
    betas = list(1.0 / np.geomspace(0.9, 2.0, 32))
    reals = (5, 31 * 32 + 26)

    def oracle_runs():
        out = []
        for r in reals:
            J = oracle.ea_couplings(3, L, r, seed)
            s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(a, r >> 5, t), bit=r & 31)
                                    for t in range(32)]) for a in range(2)]).copy()
            lab = np.tile(np.arange(32, dtype=np.int32), (2, 1))
            Es, Qs, acc, _ = oracle.omp_pt_run(3, L, s, betas, seed, r, r >> 5, 0, n, 1, J=J, labels=lab)
            out.append((s, Es, Qs, lab))
        return out

    with ThreadPoolExecutor(1) as ex:  # the oracle's C calls run while the GPU works
        fut = ex.submit(oracle_runs)
        lat = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=1024, n_temps=32, n_sets=2, seed=seed)
        ser = {"E": torch.zeros(n * 2 * 32 * 1024, dtype=torch.int64, device="cuda"),
               "Q": torch.zeros(n * 32 * 1024, dtype=torch.int64, device="cuda")}
        labels = lat.slot_labels()
        sp.batch_run([lat.batch_item(betas, ser, labels=labels)], n, 1, 1)
        lat.sync()
        assert lat.sweeps_done == n and lat.pt_steps_done == n
        got = lat.unpack()
        E = ser["E"].view(n, 2, 32, 1024)
        Q = ser["Q"].view(n, 32, 1024)
        for r, (s, Es, Qs, lab) in zip(reals, fut.result()):
            assert np.array_equal(got[:, :, r].cpu().numpy(), s), r
            assert np.array_equal(E[:, :, :, r].cpu().numpy(), Es), r
            assert np.array_equal(Q[:, :, r].cpu().numpy(), Qs), r
            assert np.array_equal(labels[:, :, r].cpu().numpy(), lab), r


@pytest.mark.parametrize("variant", [0, 2])
def test_heis_L128_one_sweep_full_lattice(variant):
    """3D Heisenberg L=128 (2M sites): one sweep from a common FP32 start,
    every site within 1e-5 of the FP64 oracle except flagged near-ties."""
    L, seed, beta = 128, 6, 0.693
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=seed)
    lat.set_variant(variant)
    s0 = oracle.heis_init(3, L, seed, 0).astype(np.float32)
    dev = np.zeros((L ** 3, 4), np.float32)
    dev[:, :3] = s0
    lat.spins.copy_(torch.from_numpy(dev.ravel()))
    lat.sweep([beta], 1)
    got = lat.spins.view(-1, 4)[:, :3].cpu().numpy()
    ref = s0.astype(np.float64)
    margin = oracle.heis_sweep(3, L, ref, beta, seed, 0, 0, want_margin=True)
    err = np.max(np.abs(got - ref), axis=1)
    flagged = margin < 1e-5
    idx = np.arange(L ** 3)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    near = flagged.copy()
    for d in (1, -1):
        for sh in ((x + d) % L + L * y + L * L * z, x + L * ((y + d) % L) + L * L * z,
                   x + L * y + L * L * ((z + d) % L)):
            near |= flagged[sh]
    assert not ((err > 1e-5) & ~near).any()
    assert (err > 1e-5).sum() <= 40


def test_heis_L128_renormalisation():
    L = 128
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=7)
    lat.sweep([0.693], 100)
    v = lat.spins.view(-1, 4)[:, :3].double()
    assert torch.max(torch.abs(torch.linalg.norm(v, dim=1) - 1)).item() <= 1e-6


def test_heis_L128_long_run_energy_matches_fp64_oracle():
    """The 3D Heisenberg configuration at full size: L = 128, beta = 0.693,
    2000 sweeps from the hot start with renormalisation every 100 sweeps, E
    every 10 sweeps.  The FP32 GPU chain and the FP64 oracle chain (same
    seed, so the same random numbers; they part at the first decision that
    differs) have window means of the energy per spin within 3 combined
    standard errors, and their paired difference has mean zero within 3
    standard errors."""
    from concurrent.futures import ThreadPoolExecutor
    L, beta, n, every, seed = 128, 0.693, 2000, 10, 10
    N = L ** 3
    lid = oracle.lattice_id(0, 0, 0)

    def oracle_run():
        s = oracle.heis_init(3, L, seed, lid)
        E, _ = oracle.omp_heis_run(3, L, s, beta, seed, lid, 0, n, renorm_every=100, measure_every=every)
        return E / N, s

    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle_run)
        lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=seed)
        out = lat.run([beta], n, measure_every=every)
        eg = out["Ef"].cpu().numpy() / N
        v = lat.spins.view(-1, 4)[:, :3].double()
        norm_dev = torch.max(torch.abs(torch.linalg.norm(v, dim=1) - 1)).item()
        eo, so = fut.result()
    assert eg.shape == eo.shape == (n // every,)
    assert norm_dev <= 1e-6  # the last sweep (2000) renormalised
    assert np.max(np.abs(np.linalg.norm(so, axis=1) - 1)) < 1e-12
    w = slice(50, None)  # sweeps 500 .. 2000
    mg, sg = binned_mean(eg[w], 15)
    mo, sob = binned_mean(eo[w], 15)
    assert abs(mg - mo) <= 3 * math.sqrt(sg ** 2 + sob ** 2) + 1e-9, (mg, sg, mo, sob)
    md, sd = binned_mean(eg[w] - eo[w], 15)
    assert abs(md) <= 3 * sd + 1e-9, (md, sd)
    assert abs(eg[0] - eo[0]) < 1e-3  # the first measurement, before the chains have drifted apart


def test_heis_long_run_energy_matches_fp64_oracle():
    """Long-run energy per spin of the FP32 GPU chain and of the FP64 oracle
    chain (same seed; they decorrelate after the first decision that differs)
    agree within 3 combined standard errors."""
    L, beta, n, seed = 12, 0.693, 3000, 8
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=seed)
    out = lat.run([beta], n, measure_every=1)
    eg = out["Ef"].cpu().numpy() / L ** 3
    s = oracle.heis_init(3, L, seed, 0)
    eo, _ = oracle.heis_run(3, L, s, beta, seed, 0, 0, n)
    eo = eo / L ** 3
    mg, sg = binned_mean(eg[300:], 30)
    mo, so = binned_mean(eo[300:], 30)
    assert abs(mg - mo) <= 3 * math.sqrt(sg ** 2 + so ** 2) + 1e-12, (mg, sg, mo, so)


def test_uneven_batch_equals_per_handle_runs():
    """An uneven batch in one launch: EA lattices of L = 8, 12, 16 and 24
    (different slot counts) and 2D Ising lattices of L = 256 and 512."""
    specs = [("ea", 8, 64, 6), ("ea", 12, 32, 5), ("ea", 16, 32, 4), ("ea", 24, 32, 3),
             ("is", 256, 1, 1), ("is", 512, 1, 1)]

    def make(k, spec):
        kind, L, n_real, n_t = spec
        if kind == "ea":
            lat = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=n_real, n_temps=n_t, n_sets=2, seed=40 + k)
            return lat, list(1.0 / np.geomspace(0.8, 2.2, n_t))
        return sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=40 + k), [0.4407]

    n = 7
    batch = [make(k, s) for k, s in enumerate(specs)]
    plain = [make(k, s) for k, s in enumerate(specs)]
    items, sers = [], []
    for lat, betas in batch:
        ser = lat.series_buffers(n)
        if lat.n_sets < 2:
            ser.pop("Q", None)
        sers.append(ser)
        items.append(lat.batch_item(betas, ser))
    sp.batch_run(items, n, 1, 1)
    batch[0][0].sync()
    for (lb, _), (lp, betas), ser in zip(batch, plain, sers):
        out = lp.run(betas, n, 1, 1)
        assert torch.equal(lb.spins, lp.spins)
        for key in ser:
            assert torch.equal(ser[key], out[key]), key


UNEVEN_EA = [(8, 512, 24), (12, 256, 30), (16, 128, 36), (24, 64, 42), (32, 32, 48)]
UNEVEN_ISING = [256, 512, 1024, 2048, 4096]


@pytest.mark.parametrize("ising_layout", [B.SPIN_I8, B.SPIN_MSC1])
def test_uneven_batch_full_size(ising_layout):
    """The full uneven batch (EA L = 8..32 with 512..32 realisations and
    24..48 temperatures in [0.8, 2.2], two sets; 2D Ising L = 256..4096, int8
    or coded) in one batched launch, measurement and exchange every sweep:
    equal to plain per-handle runs over the configuration's 50 sweeps, and
    one sampled realisation of every EA size equal to the oracle."""
    n = 50

    def build():
        side = []
        for k, (L, R, T) in enumerate(UNEVEN_EA):
            lat = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=R, n_temps=T, n_sets=2, seed=50 + k)
            side.append((lat, list(1.0 / np.geomspace(0.8, 2.2, T))))
        for k, L in enumerate(UNEVEN_ISING):
            side.append((sp.Lattice(B.SPIN_ISING, 2, L, ising_layout, seed=60 + k), [0.4407]))
        return side

    batch, plain = build(), build()
    items, sers = [], []
    for lat, betas in batch:
        ser = lat.series_buffers(n)
        if lat.n_sets < 2:
            ser.pop("Q", None)
        sers.append(ser)
        items.append(lat.batch_item(betas, ser))
    sp.batch_run(items, n, 1, 1)
    batch[0][0].sync()
    for (lb, _), (lp, betas), ser in zip(batch, plain, sers):
        out = lp.run(betas, n, 1, 1 if lp.model == B.SPIN_EA else 0)
        assert torch.equal(lb.spins, lp.spins), lb.L
        for key in ser:
            assert torch.equal(ser[key], out[key]), (lb.L, key)
    for (lat, betas), (L, R, T), r in zip(batch, UNEVEN_EA, (511, 200, 64, 33, 31)):
        s, Es, Qs = _uneven_oracle(L, T, r, lat.seed, tuple(betas), n)
        got = lat.unpack()[:, :, r].cpu().numpy()
        assert np.array_equal(got, s), L
        ser = sers[UNEVEN_EA.index((L, R, T))]
        assert np.array_equal(ser["E"].view(n, 2, T, R)[:, :, :, r].cpu().numpy(), Es), L
        assert np.array_equal(ser["Q"].view(n, T, R)[:, :, r].cpu().numpy(), Qs), L


_UNEVEN_CACHE = {}


def _uneven_oracle(L, T, r, seed, betas, n):
    """Oracle tempering run of realisation r of an uneven-batch EA lattice
    (cached: both Ising layouts of the test share the EA lattices)."""
    key = (L, T, r, seed, betas, n)
    if key not in _UNEVEN_CACHE:
        J = oracle.ea_couplings(3, L, r, seed)
        s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(a, r >> 5, t), bit=r & 31)
                                for t in range(T)]) for a in range(2)]).copy()
        Es, Qs, _, _ = oracle.omp_pt_run(3, L, s, list(betas), seed, r, r >> 5, 0, n, 1, J=J)
        _UNEVEN_CACHE[key] = (s, Es, Qs)
    return _UNEVEN_CACHE[key]


def _tab_rng_e():
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    for line in open(os.path.join(here, "golden", "tab_rng_exact.txt")):
        if line.strip() and not line.startswith("#"):
            return float(line.split()[2])


@pytest.mark.parametrize("order", [B.SPIN_ORDER_DCB, B.SPIN_ORDER_DCB_SYMMETRIC])
def test_dcb_L16384_energy_matches_exact(order):
    """The double-checkerboard chain on the full L = 16384 lattice (tile 64,
    10 hits) at beta = 0.4 samples the exact energy per spin (Tab. rng; at
    this beta the L = 1024 torus value equals the infinite lattice's to far
    below the statistical error of 2^28 spins)."""
    L, T, k = 16384, 64, 10
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=91)
    lat.set_update_order(order, T, k)
    lat.sweep([0.4], 300)
    out = lat.run([0.4], 600, measure_every=k)
    e = -out["E"].cpu().numpy().astype(np.float64) / L ** 2
    m, s = binned_mean(e, 20)
    assert abs(m - _tab_rng_e()) <= 4 * s + 1e-6, (m, s)


def test_ea_w64_full_size_batched_equals_plain():
    """3D EA L = 16, 1024 realisations x 32 slots x 2 sets, w = 64: the
    batched launch equals the per-handle pair kernel, series included."""
    L, n = 16, 4
    betas = list(1.0 / np.geomspace(0.9, 2.0, 32))
    a = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=1024, n_temps=32, n_sets=2, seed=5)
    b = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=1024, n_temps=32, n_sets=2, seed=5)
    a.set_msc_width(64)
    b.set_msc_width(64)
    ser = a.series_buffers(n)
    sp.batch_run([a.batch_item(betas, ser)], n, 1, 1)
    out = b.run(betas, n, 1, 1)
    a.sync()
    assert torch.equal(a.spins, b.spins)
    for key in ("E", "M", "Q"):
        assert torch.equal(ser[key], out[key]), key


def test_slabs_L16384_equal_unsplit():
    """Four slabs of the L = 16384 lattice with ghost rows exchanged on the
    device equal the unsplit sweep."""
    from paper_1101_1427_gb300 import slab as S
    L, P, n, beta, seed = 16384, 4, 2, 0.4407, 93
    full = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
    parts = [S.split_rows(L, P, k) for k in range(P)]
    slabs = []
    for y0, rows in parts:
        sl = torch.empty(rows + 2, L, dtype=torch.int8, device="cuda")
        sl[1:rows + 1] = full.spins.view(L, L)[y0:y0 + rows]
        slabs.append(sl)
    full.sweep([beta], n)
    for sweep in range(n):
        for colour in (0, 1):
            S.exchange_ghosts_local(slabs)
            for (y0, rows), sl in zip(parts, slabs):
                S.phase(sl, L, y0, rows, beta, seed, 0, sweep, colour)
    for (y0, rows), sl in zip(parts, slabs):
        assert torch.equal(sl[1:rows + 1], full.spins.view(L, L)[y0:y0 + rows]), y0
