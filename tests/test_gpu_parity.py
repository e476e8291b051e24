"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on the
same seeded inputs.  Ising / EA lattices, energies, magnetisations, overlaps
and exchange decisions are compared bit for bit; Heisenberg spins within the
stated FP32 tolerances."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# ------------------------------------------------------------------ Philox
@pytest.mark.parametrize("tag,colour,extra,lid,sweep", [
    (0, 0, 0, 0, 0), (0, 1, 0, 0x01002003, 7), (1, 0, 5, 12, 0), (3, 0, 0, 0xFFFFFF, 2 ** 31 + 5),
    (4, 1, (1 << 27) - 1, 99, 123456)])
def test_rng_matches_oracle(tag, colour, extra, lid, sweep):
    seed = 0x9E3779B97F4A7C15
    count = 4099  # ragged tail
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    B.spin_rng_fill(seed, tag, colour, extra, lid, sweep, count, out)
    got = host(out).view(np.uint32)
    for idx in list(range(16)) + [1000, 1001, 4095, 4096, 4097, 4098]:
        assert got[idx] == oracle.draw(seed, tag, colour, extra, lid, sweep, idx), idx


# ------------------------------------------------------------------ Ising, int8
def oracle_lattices_ising(dim, L, seed, n_real, n_temps, n_sets, ea=False):
    out = np.zeros((n_sets, n_temps, n_real, L ** dim), np.int8)
    for a in range(n_sets):
        for t in range(n_temps):
            for r in range(n_real):
                lid = oracle.lattice_id(a, (r >> 5) if ea else r, t)
                out[a, t, r] = oracle.ising_init(dim, L, seed, lid, bit=(r & 31) if ea else 0)
    return out


@pytest.mark.parametrize("dim,L,n_real,n_temps", [(2, 64, 1, 1), (2, 6, 2, 3), (3, 8, 1, 2), (3, 10, 3, 1)])
def test_ising_init_matches_oracle(dim, L, n_real, n_temps):
    lat = sp.Lattice(B.SPIN_ISING, dim, L, B.SPIN_I8, n_real=n_real, n_temps=n_temps, seed=77)
    got = host(lat.spins).reshape(1, n_temps, n_real, -1)
    assert np.array_equal(got, oracle_lattices_ising(dim, L, 77, n_real, n_temps, 1))


def _ising_run_oracle(dim, L, seed, betas, n_real, n_sweeps, first=0):
    n_temps = len(betas)
    s = oracle_lattices_ising(dim, L, seed, n_real, n_temps, 1)
    E = np.zeros((n_sweeps, n_temps, n_real), np.int64)
    M = np.zeros((n_sweeps, n_temps, n_real), np.int64)
    for t in range(n_temps):
        for r in range(n_real):
            e, m, _ = oracle.ising_run(dim, L, s[0, t, r], betas[t], seed,
                                       oracle.lattice_id(0, r, t), first, n_sweeps)
            E[:, t, r], M[:, t, r] = e, m
    return s, E, M


@pytest.mark.parametrize("L,n_real,calls", [(256, 1, (4,)), (512, 3, (3, 5)), (768, 2, (9, 1, 4))])
def test_ising2d_i8_coded_variant_bit_exact(L, n_real, calls):
    """int8 ferromagnets with L % 256 == 0 sweep through the 1-bit coded
    layout (variant 4, the default there) in calls of >= 4 sweeps and through
    the fused pass otherwise; lattices, E and M equal the oracle after every
    call, so packing, the coded sweeps and unpacking are exact."""
    seed, betas = 13, [0.4407]
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=n_real, seed=seed)
    assert B.lib().spin_set_variant(lat.h, 4) == B.SPIN_OK
    s = oracle_lattices_ising(2, L, seed, n_real, 1, 1)
    done = 0
    for n in calls:
        lat.sweep(betas, n)
        for r in range(n_real):
            E, M, _ = oracle.ising_run(2, L, s[0, 0, r], betas[0], seed, oracle.lattice_id(0, r, 0), done, n)
        done += n
        assert np.array_equal(host(lat.spins).reshape(s.shape), s), (L, n)
        Eg, Mg, _ = lat.measure()
        assert np.array_equal(host(Eg), [oracle.ising_energy(2, L, s[0, 0, r]) for r in range(n_real)])
        assert np.array_equal(host(Mg), [int(s[0, 0, r].astype(np.int64).sum()) for r in range(n_real)])


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_ising2d_L64_1000_sweeps_bit_exact(variant):
    """2D Ising L=64, beta = 0.4407, 1000 sweeps, E and M after every sweep."""
    L, seed, beta, n = 64, 1, 0.4407, 1000
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
    lat.set_variant(variant)
    out = lat.run([beta], n, measure_every=1)
    s, E, M = _ising_run_oracle(2, L, seed, [beta], 1, n)
    assert np.array_equal(host(out["E"]), E.ravel())
    assert np.array_equal(host(out["M"]), M.ravel())
    assert np.array_equal(host(lat.spins), s.ravel())
    assert lat.sweeps_done == n


@pytest.mark.parametrize("dim,L,betas,n_real,variant", [
    (2, 6, [0.3, 0.44], 2, 0),        # generic kernel, L % 8 != 0
    (2, 24, [0.5], 1, 0),             # 2D kernel, L % 16 != 0
    (2, 48, [0.4, 0.45, 0.9], 2, 1),  # fused kernel, several lattices, ragged strips
    (2, 32, [0.0, 5.0], 1, 1),        # infinite and (near) zero temperature
    (2, 8, [0.3, 0.44], 2, 3),        # resident kernel, one chunk per row
    (2, 24, [0.5, 0.0], 1, 3),        # resident kernel, three chunks per row
    (2, 80, [0.44, 0.3], 1, 3),       # resident kernel, two chunks per thread
    (2, 128, [0.4407, 5.0], 2, 3),    # resident kernel, largest lattice (four chunks per thread)
    (3, 8, [0.22, 0.3], 1, 0),        # 3D chunk kernel, one chunk per row
    (3, 16, [0.0, 0.2216, 50.0], 2, 0),  # 3D chunk kernel, degenerate temperatures
    (3, 24, [0.25], 1, 0),            # 3D chunk kernel, odd number of chunks per row
    (3, 8, [0.22, 0.3], 2, 3),        # 3D resident kernel, one chunk per row
    (3, 16, [0.0, 0.2216, 50.0], 1, 3),  # 3D resident kernel, degenerate temperatures
    (3, 24, [0.25], 1, 3),            # 3D resident kernel, four chunks per thread
    (3, 12, [0.25], 2, 0)])           # generic kernel (L % 8 != 0)
def test_ising_sweeps_bit_exact(dim, L, betas, n_real, variant):
    seed, n = 5, 13
    lat = sp.Lattice(B.SPIN_ISING, dim, L, B.SPIN_I8, n_real=n_real, n_temps=len(betas), seed=seed)
    lat.set_variant(variant)
    lat.sweep(betas, 5)
    lat.sweep(betas, 8)  # continues the chain
    s, E, M = _ising_run_oracle(dim, L, seed, betas, n_real, n)
    assert np.array_equal(host(lat.spins), s.ravel())
    Eg, Mg, _ = lat.measure()
    assert np.array_equal(host(Eg), E[-1].ravel()) and np.array_equal(host(Mg), M[-1].ravel())


def test_resident_long_call_equals_phases_and_oracle():
    """5000 sweeps in one call: the resident kernel splits them over two
    launches (at most 4096 sweeps each); the lattices equal those of the
    in-place phases and of the oracle."""
    L, seed, n = 16, 9, 5000
    betas = [0.35, 0.4407, 0.6]
    a = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=3, seed=seed)
    b = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=3, seed=seed)
    a.set_variant(0)
    assert b.sweeps_done == 0
    a.sweep(betas, n)
    b.sweep(betas, n)  # default variant for L <= 128: resident
    torch.cuda.synchronize()
    assert torch.equal(a.spins, b.spins)
    s, _, _ = _ising_run_oracle(2, L, seed, betas, 1, n)
    assert np.array_equal(host(b.spins), s.ravel())


def test_fused_equals_phases_on_large_lattice():
    L, seed = 4096, 3
    a = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
    b = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
    a.set_variant(0)
    b.set_variant(1)
    a.sweep([0.4407], 3)
    b.sweep([0.4407], 3)
    torch.cuda.synchronize()
    assert torch.equal(a.spins, b.spins)


def test_fused_many_lattices_short_strips():
    """20 int8 lattices of L = 2048 (the tempering benchmark's shape): the
    fused sweep splits each lattice into many short strips (a ragged last
    one included); sampled lattices equal the oracle."""
    L, seed, n = 2048, 71, 3
    betas = list(np.linspace(0.1, 0.15, 20))
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=20, seed=seed)
    lat.set_variant(1)
    lat.sweep(betas, n)
    got = host(lat.spins).reshape(20, -1)
    for t in (0, 19):
        lid = oracle.lattice_id(0, 0, t)
        s = oracle.ising_init(2, L, seed, lid)
        oracle.ising_run(2, L, s, betas[t], seed, lid, 0, n, series=False)
        assert np.array_equal(got[t], s), t


# ------------------------------------------------------------------ EA
def _ea_oracle(L, seed, betas, n_real, n_sets, n_sweeps, pt_every=0, reals=None, width=32, dim=3,
               labels=None):
    """Oracle runs of single realisations; `width` realisations share each
    update uniform (key r >> 5 for 32, r >> 6 for 64).  labels (optional,
    int32 [n_sets, n_temps, n_real], modified in place) are moved with the
    configurations as the oracle exchanges them."""
    n_temps = len(betas)
    shift = 5 if width == 32 else 6
    reals = range(n_real) if reals is None else reals
    res = {}
    for r in reals:
        J = oracle.ea_couplings(dim, L, r, seed)
        sp_ = np.stack([np.stack([oracle.ising_init(dim, L, seed, oracle.lattice_id(a, r >> 5, t),
                                                    bit=r & 31) for t in range(n_temps)])
                        for a in range(n_sets)]).copy()
        lab = None if labels is None else np.ascontiguousarray(labels[:, :, r])
        E, Q, acc, _ = oracle.pt_run(dim, L, sp_, betas, seed, r, r >> shift, 0, n_sweeps, pt_every, J=J,
                                     labels=lab)
        if labels is not None:
            labels[:, :, r] = lab
        res[r] = (J, sp_, E, Q, acc)
    return res


@pytest.mark.parametrize("L,width", [(16, 32), (10, 32), (16, 64)])
def test_ea2d_coded_bit_exact(L, width):
    """The coded EA glass on the square lattice (the paper's Sec. 5 benchmark
    is 2D): exchange and E, M, Q every sweep, vectorised (L % 8 == 0) and
    per-site (L = 10) paths, w = 32 and 64; sampled realisations equal the
    oracle (int8 per realisation, four bonds)."""
    seed, n_real, n = 31, 128, 8
    betas = list(1.0 / np.geomspace(0.8, 3.0, 5))
    lat = sp.Lattice(B.SPIN_EA, 2, L, B.SPIN_MSC1, n_real=n_real, n_temps=5, n_sets=2, seed=seed)
    if width == 64:
        lat.set_msc_width(64)
    acc = torch.zeros(10, dtype=torch.int64, device="cuda")
    out = lat.run(betas, n, measure_every=1, pt_every=1, accepted=acc)
    got = host(lat.unpack())
    E = host(out["E"]).reshape(n, 2, 5, n_real)
    Q = host(out["Q"]).reshape(n, 5, n_real)
    _, M_now, _ = lat.measure()  # of the final state (the series precede each sweep's exchange)
    M_now = host(M_now).reshape(2, 5, n_real)
    ref = _ea_oracle(L, seed, betas, n_real, 2, n, pt_every=1, reals=(0, 33, 64, 127), width=width, dim=2)
    for r, (J, s, Es, Qs, ac) in ref.items():
        assert np.array_equal(got[:, :, r], s), r
        assert np.array_equal(E[:, :, :, r], Es), r
        assert np.array_equal(Q[:, :, r], Qs), r
        assert np.array_equal(M_now[:, :, r], s.astype(np.int64).sum(axis=2)), r
    # the couplings equal the oracle's draws (bit r of group r >> 5)
    Jw = host(lat.couplings).view(np.uint32).reshape(n_real // 32, 2, 2, L * L // 2)
    for r in (0, 127):
        Jo = oracle.ea_couplings(2, L, r, seed).reshape(2, L * L)
        for d in range(2):
            for i in (0, 1, L + 1, L * L - 1):
                c = ((i % L) + (i // L)) & 1
                assert ((Jw[r >> 5, d, c, i >> 1] >> (r & 31)) & 1) == (Jo[d, i] < 0), (r, d, i)


@pytest.mark.parametrize("L,T", [(8, 4), (6, 4), (8, 6)])
def test_ea_w64_shared_uniforms_bit_exact(L, T):
    """w = 64 (Sec. 5): realisations r and r' with r >> 6 == r' >> 6 share
    every update uniform; plain per-handle path with exchange and
    measurement every sweep, sampled realisations of both words of a pair.
    T = 6 leaves the second block of four slots of a thread half empty."""
    seed, n_real, n = 23, 128, 10
    betas = list(1.0 / np.geomspace(0.9, 2.0, T))
    lat = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=n_real, n_temps=T, n_sets=2, seed=seed)
    lat.set_msc_width(64)
    out = lat.run(betas, n, measure_every=1, pt_every=1)
    got = host(lat.unpack())
    E = host(out["E"]).reshape(n, 2, T, n_real)
    Q = host(out["Q"]).reshape(n, T, n_real)
    ref = _ea_oracle(L, seed, betas, n_real, 2, n, pt_every=1, reals=(0, 31, 32, 63, 64, 127), width=64)
    for r, (J, s, Es, Qs, ac) in ref.items():
        assert np.array_equal(got[:, :, r], s), r
        assert np.array_equal(E[:, :, :, r], Es), r
        assert np.array_equal(Q[:, :, r], Qs), r
    # and w = 32 gives a different chain from the same start
    lat32 = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=n_real, n_temps=T, n_sets=2, seed=seed)
    lat32.run(betas, n, measure_every=0, pt_every=1, series=False)
    assert not torch.equal(lat32.spins, lat.spins)


@pytest.mark.parametrize("layout", [B.SPIN_I8, B.SPIN_MSC1])
def test_ea_couplings_and_init_match_oracle(layout):
    L, seed, n_real = 6, 11, 64
    lat = sp.Lattice(B.SPIN_EA, 3, L, layout, n_real=n_real, n_temps=2, n_sets=2, seed=seed)
    got = host(lat.unpack())
    exp = oracle_lattices_ising(3, L, seed, n_real, 2, 2, ea=True)
    assert np.array_equal(got, exp)
    if layout == B.SPIN_I8:
        Jg = host(lat.couplings).reshape(n_real, -1)
        for r in (0, 1, 31, 32, 63):
            assert np.array_equal(Jg[r], oracle.ea_couplings(3, L, r, seed))
    else:
        N = L ** 3
        Jw = host(lat.couplings).view(np.uint32).reshape(n_real // 32, 3, N)
        i = np.arange(N)
        colour = (i % L + (i // L) % L + i // (L * L)) % 2
        slot = colour * (N // 2) + (i >> 1)  # colour-split storage of bond (i, i + e_d)
        for r in (0, 5, 31, 32, 63):
            bits = ((Jw[r >> 5][:, slot] >> np.uint32(r & 31)) & 1).astype(np.int8).ravel()
            assert np.array_equal(1 - 2 * bits, oracle.ea_couplings(3, L, r, seed))


@pytest.mark.parametrize("layout,L", [(B.SPIN_I8, 6), (B.SPIN_MSC1, 6), (B.SPIN_MSC1, 8)])
def test_ea_sweeps_measure_bit_exact(layout, L):
    seed, n_real, betas, n = 13, 64, [0.9, 1.3, 2.0], 6
    lat = sp.Lattice(B.SPIN_EA, 3, L, layout, n_real=n_real, n_temps=3, n_sets=2, seed=seed)
    lat.sweep(betas, n)
    E, M, Q = lat.measure()
    got = host(lat.unpack())
    E, M, Q = host(E).reshape(2, 3, n_real), host(M).reshape(2, 3, n_real), host(Q).reshape(3, n_real)
    ref = _ea_oracle(L, seed, betas, n_real, 2, n, reals=[0, 1, 30, 31, 32, 47, 63])
    for r, (J, s, Es, Qs, _) in ref.items():
        assert np.array_equal(got[:, :, r], s), r
        assert np.array_equal(E[:, :, r], Es[-1]), r
        assert np.array_equal(Q[:, r], Qs[-1]), r
        for a in range(2):
            for t in range(3):
                assert M[a, t, r] == s[a, t].sum()


@pytest.mark.parametrize("layout,L", [(B.SPIN_I8, 4), (B.SPIN_MSC1, 4), (B.SPIN_I8, 6), (B.SPIN_MSC1, 6)])
def test_ea_parallel_tempering_bit_exact(layout, L):
    """L = 6: int8 lattices of 216 bytes, not a multiple of 16."""
    seed, n_real, n = 21, 32, 40
    betas = list(1.0 / np.geomspace(0.9, 2.0, 5))
    lat = sp.Lattice(B.SPIN_EA, 3, L, layout, n_real=n_real, n_temps=5, n_sets=2, seed=seed)
    acc = torch.zeros(2 * 5, dtype=torch.int64, device="cuda")
    # configuration labels: arbitrary caller values, moved with the configurations
    lab0 = (np.arange(2 * 5 * n_real, dtype=np.int32) * 7 + 3).reshape(2, 5, n_real)
    labels = torch.from_numpy(lab0.copy()).cuda()
    out = lat.run(betas, n, measure_every=1, pt_every=1, accepted=acc, labels=labels)
    got = host(lat.unpack())
    Eser = host(out["E"]).reshape(n, 2, 5, n_real)
    Qser = host(out["Q"]).reshape(n, 5, n_real)
    lab_ref = lab0.copy()
    ref = _ea_oracle(L, seed, betas, n_real, 2, n, pt_every=1, labels=lab_ref)
    acc_ref = np.zeros((2, 5), np.int64)
    for r, (J, s, Es, Qs, ac) in ref.items():
        assert np.array_equal(got[:, :, r], s), r
        assert np.array_equal(Eser[:, :, :, r], Es), r
        assert np.array_equal(Qser[:, :, r], Qs), r
        acc_ref += ac
    assert np.array_equal(host(acc).reshape(2, 5), acc_ref)
    assert np.array_equal(host(labels), lab_ref)
    assert not np.array_equal(lab_ref, lab0)
    assert acc_ref.sum() > 0
    assert lat.pt_steps_done == n


def test_msc_equals_int8_ea():
    L, seed, n_real, betas = 8, 4, 64, [1.0, 1.5]
    a = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_I8, n_real=n_real, n_temps=2, n_sets=2, seed=seed)
    b = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=n_real, n_temps=2, n_sets=2, seed=seed)
    for lat in (a, b):
        lat.run(betas, 25, pt_every=1)
    assert torch.equal(a.unpack(), b.unpack())


# ------------------------------------------------------------------ 2D coded ferromagnet
@pytest.mark.parametrize("L,betas", [(256, [0.4407]), (512, [0.4, 0.5])])
def test_msc2d_bit_exact(L, betas):
    seed, n = 9, 7
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=len(betas), seed=seed)
    assert np.array_equal(host(lat.unpack()).reshape(len(betas), -1),
                          oracle_lattices_ising(2, L, seed, 1, len(betas), 1).reshape(len(betas), -1))
    lat.sweep(betas, n)
    s, E, M = _ising_run_oracle(2, L, seed, betas, 1, n)
    assert np.array_equal(host(lat.unpack()).ravel(), s.ravel())
    Eg, Mg, _ = lat.measure()
    assert np.array_equal(host(Eg), E[-1].ravel()) and np.array_equal(host(Mg), M[-1].ravel())


def test_msc2d_pack_roundtrip():
    L = 256
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, seed=2)
    x = torch.where(torch.rand(L * L, device="cuda") < 0.5, -1, 1).to(torch.int8)
    lat.pack(x)
    assert torch.equal(lat.unpack().view(-1), x)


# ------------------------------------------------------------------ Heisenberg
def test_heis_init_close_to_oracle():
    L = 8
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=3)
    got = host(lat.spins).reshape(-1, 4)
    ref = oracle.heis_init(3, L, 3, oracle.lattice_id(0, 0, 0))
    assert np.max(np.abs(got[:, :3] - ref)) < 1e-6 and np.all(got[:, 3] == 0)


@pytest.mark.parametrize("variant", [0, 2])
def test_heis_one_sweep_within_tolerance(variant):
    """Same FP32 start for both; after one sweep every site agrees to 1e-5,
    except sites whose accept/reject margin |u3 - exp(-beta dE)| is below 1e-5
    in the FP64 oracle and the later-updated neighbours of such sites."""
    L, seed, beta = 16, 8, 0.693
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=seed)
    lat.set_variant(variant)
    s0 = oracle.heis_init(3, L, seed, 0).astype(np.float32)
    dev = np.zeros((L ** 3, 4), np.float32)
    dev[:, :3] = s0
    lat.spins.copy_(torch.from_numpy(dev.ravel()))
    lat.sweep([beta], 1)
    got = host(lat.spins).reshape(-1, 4)[:, :3]
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
    bad = (err > 1e-5) & ~near
    assert not bad.any(), (np.nonzero(bad)[0][:10], err[bad][:10])
    assert (err > 1e-5).sum() <= 20


@pytest.mark.parametrize("variant", [0, 2])
def test_heis_renormalisation_bound(variant):
    L = 16
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=4)
    lat.set_variant(variant)
    lat.sweep([0.693], 100)
    v = host(lat.spins).reshape(-1, 4)[:, :3].astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(v, axis=1) - 1)) <= 1e-6


def test_heis_measure_matches_oracle_on_oracle_state():
    L = 12
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, n_temps=2, seed=5)
    states = [oracle.heis_init(3, L, 5 + k, 0).astype(np.float32).astype(np.float64) for k in range(2)]
    dev = np.zeros((2, L ** 3, 4), np.float32)
    for k in range(2):
        dev[k, :, :3] = states[k]
    lat.spins.copy_(torch.from_numpy(dev.ravel()))
    Ef, Mf = lat.measure()
    Ef, Mf = host(Ef), host(Mf)
    for k in range(2):
        assert abs(Ef[k] - oracle.heis_energy(3, L, states[k])) < 1e-9 * L ** 3
        assert np.allclose(Mf[k], oracle.heis_magnetisation(3, L, states[k]), atol=1e-9 * L ** 3)


def test_ising_measure_on_oracle_state():
    L = 20
    lat = sp.Lattice(B.SPIN_ISING, 3, L, B.SPIN_I8, seed=5)
    s = oracle.ising_init(3, L, 99, 0)
    lat.spins.copy_(torch.from_numpy(s))
    E, M, _ = lat.measure()
    assert host(E)[0] == oracle.ising_energy(3, L, s) and host(M)[0] == s.sum()


# ------------------------------------------------------------------ errors
def test_invalid_arguments_are_rejected():
    with pytest.raises(B.SpinError):
        sp.Lattice(B.SPIN_ISING, 2, 63, B.SPIN_I8)
    with pytest.raises(B.SpinError):
        sp.Lattice(B.SPIN_EA, 3, 8, B.SPIN_MSC1, n_real=20)
    lat = sp.Lattice(B.SPIN_ISING, 2, 16, B.SPIN_I8, seed=1)
    with pytest.raises(B.SpinError):
        lat.sweep([float("nan")])
    with pytest.raises(B.SpinError):
        B.spin_sweep(lat.h, None, [0.4], 1, 2)  # wrong seed
    with pytest.raises(B.SpinError):
        lat.sweep([-0.1])
    lat.sync()


@pytest.mark.parametrize("dim,L", [(2, 16), (3, 8)])
def test_resident_two_replica_sets_equal_phases(dim, L):
    """Two replica sets x 2 realisations x 3 slots: the resident kernel
    (variant 3) keys every lattice as the colour phases do, sweeps alone and
    in runs that measure E and M in place or, with the overlap requested,
    through the separate measurement; both sides equal, E and M included."""
    seed, betas, n = 41, [0.25, 0.44, 0.7], 7
    a = sp.Lattice(B.SPIN_ISING, dim, L, B.SPIN_I8, n_real=2, n_temps=3, n_sets=2, seed=seed)
    b = sp.Lattice(B.SPIN_ISING, dim, L, B.SPIN_I8, n_real=2, n_temps=3, n_sets=2, seed=seed)
    a.set_variant(0)
    b.set_variant(3)
    a.sweep(betas, 3)
    b.sweep(betas, 3)
    oa, ob = a.run(betas, n, measure_every=2), b.run(betas, n, measure_every=2)
    for key in ("E", "M", "Q"):
        assert torch.equal(oa[key], ob[key]), key
    # E and M only: the resident side measures in place
    ser = {}
    for name, lat in (("a", a), ("b", b)):
        E = torch.zeros(4 * lat.n_lat, dtype=torch.int64, device="cuda")  # ceil(n / 2) rows
        M = torch.zeros(4 * lat.n_lat, dtype=torch.int64, device="cuda")
        B.spin_run(lat.h, None, betas, n, 2, 0, E, M, None, None, None, None)
        ser[name] = (E, M)
    assert torch.equal(ser["a"][0], ser["b"][0]) and torch.equal(ser["a"][1], ser["b"][1])
    Ea, Eb = a.measure()[0], b.measure()[0]
    assert torch.equal(a.spins, b.spins) and torch.equal(Ea, Eb)
