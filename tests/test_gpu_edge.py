"""Edge cases of the GPU path against the oracle: zero sweeps, the smallest
lattices of every model and layout, degenerate temperatures (beta = 0: every
update flips; beta large: only dE <= 0 flips) in every layout, the largest
number of lattices one launch indexes, sweep counters near 2^32, and long
multi-hit runs."""
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


@pytest.mark.parametrize("model,dim,L,layout,R,T,S", [
    (B.SPIN_ISING, 2, 16, B.SPIN_I8, 1, 2, 1), (B.SPIN_ISING, 2, 256, B.SPIN_MSC1, 1, 1, 1),
    (B.SPIN_EA, 3, 4, B.SPIN_MSC1, 32, 2, 2), (B.SPIN_EA, 3, 4, B.SPIN_I8, 3, 2, 2),
    (B.SPIN_HEISENBERG, 3, 4, B.SPIN_F32X4, 1, 1, 1)])
def test_zero_sweeps_change_nothing(model, dim, L, layout, R, T, S):
    lat = sp.Lattice(model, dim, L, layout, n_real=R, n_temps=T, n_sets=S, seed=3)
    before = lat.spins.clone()
    betas = [0.5] * T
    lat.sweep(betas, 0)
    out = lat.run(betas, 0, measure_every=1, pt_every=1 if model == B.SPIN_EA else 0)
    assert torch.equal(lat.spins, before) and lat.sweeps_done == 0 and lat.pt_steps_done == 0
    assert all(v.numel() == 0 for v in out.values())


@pytest.mark.parametrize("dim", [2, 3])
def test_smallest_ising_lattices(dim):
    """L = 4 (the smallest even lattice whose sites have distinct neighbours)."""
    L, seed, betas, n = 4, 8, [0.0, 0.3, 0.6, 50.0], 9
    lat = sp.Lattice(B.SPIN_ISING, dim, L, B.SPIN_I8, n_temps=len(betas), seed=seed)
    out = lat.run(betas, n, measure_every=1)
    E = host(out["E"]).reshape(n, len(betas))
    for t, beta in enumerate(betas):
        lid = oracle.lattice_id(0, 0, t)
        s = oracle.ising_init(dim, L, seed, lid)
        e, _, _ = oracle.ising_run(dim, L, s, beta, seed, lid, 0, n)
        assert np.array_equal(host(lat.spins).reshape(len(betas), -1)[t], s), beta
        assert np.array_equal(E[:, t], e), beta


@pytest.mark.parametrize("betas", [[0.0], [50.0], [0.0, 50.0]])
def test_coded_2d_degenerate_temperatures(betas):
    """beta = 0: every Metropolis update flips (thr = 2^32 - 1 misses only the
    word 0xFFFFFFFF); beta = 50: only dE <= 0 flips (thr = 0)."""
    L, seed, n = 256, 12, 4
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=len(betas), seed=seed)
    lat.sweep(betas, n)
    got = host(lat.unpack()).reshape(len(betas), -1)
    for t, beta in enumerate(betas):
        lid = oracle.lattice_id(0, 0, t)
        s = oracle.ising_init(2, L, seed, lid)
        for sweep in range(n):
            oracle.ising_sweep(2, L, s, beta, seed, lid, sweep)
        assert np.array_equal(got[t], s), beta


@pytest.mark.parametrize("layout", [B.SPIN_I8, B.SPIN_MSC1])
def test_ea_degenerate_temperatures_with_exchange(layout):
    """3D EA with slots at beta = 0 and beta = 50 next to ordinary ones, the
    exchange between them included."""
    L, seed, n, R = 4, 14, 6, 32
    betas = [50.0, 1.0, 0.4, 0.0]
    lat = sp.Lattice(B.SPIN_EA, 3, L, layout, n_real=R, n_temps=4, n_sets=2, seed=seed)
    out = lat.run(betas, n, measure_every=1, pt_every=1)
    got = host(lat.unpack())
    E = host(out["E"]).reshape(n, 2, 4, R)
    for r in (0, 13, 31):
        J = oracle.ea_couplings(3, L, r, seed)
        s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(a, r >> 5, t), bit=r & 31)
                                for t in range(4)]) for a in range(2)]).copy()
        Es, _, _, _ = oracle.pt_run(3, L, s, betas, seed, r, r >> 5, 0, n, 1, J=J)
        assert np.array_equal(got[:, :, r], s), r
        assert np.array_equal(E[:, :, :, r], Es), r


def test_heisenberg_smallest_lattice_and_infinite_temperature():
    """L = 4 at beta = 0: every proposal is accepted (u3 < 1 = exp(0)), so
    after one sweep every spin is its proposal; FP32 within 1e-6 of FP64."""
    L, seed = 4, 21
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=seed)
    s0 = oracle.heis_init(3, L, seed, 0).astype(np.float32)
    dev = np.zeros((L ** 3, 4), np.float32)
    dev[:, :3] = s0
    lat.spins.copy_(torch.from_numpy(dev.ravel()))
    lat.sweep([0.0], 1)
    ref = s0.astype(np.float64)
    oracle.heis_sweep(3, L, ref, 0.0, seed, 0, 0)
    got = host(lat.spins).reshape(-1, 4)[:, :3]
    assert np.max(np.abs(got - ref)) <= 1e-6
    assert not np.allclose(ref, s0)


def test_largest_lattice_count_per_launch():
    """65535 lattices (the most a launch indexes in its grid's y dimension),
    257 slots x 255 realisations of int8 L = 4: sampled lattices equal the
    oracle; 65536 are refused."""
    L, seed, n, T, R = 4, 25, 3, 257, 255
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=R, n_temps=T, seed=seed)
    betas = list(np.linspace(0.1, 0.8, T))
    lat.sweep(betas, n)
    got = host(lat.spins).reshape(T, R, -1)
    for t, r in ((0, 0), (0, 254), (128, 77), (256, 0), (256, 254)):
        lid = oracle.lattice_id(0, r, t)
        s = oracle.ising_init(2, L, seed, lid)
        for sweep in range(n):
            oracle.ising_sweep(2, L, s, betas[t], seed, lid, sweep)
        assert np.array_equal(got[t, r], s), (t, r)
    with pytest.raises(B.SpinError):
        sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_real=256, n_temps=256, seed=seed)


def test_sweep_counter_near_its_limit():
    """The sweep number is a 32-bit counter word: runs starting just below
    2^32 draw the oracle's words, and a call that would pass 2^32 - 1 is
    refused without changing anything."""
    L, seed, beta = 16, 27, 0.44
    start = 2 ** 32 - 4
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
    s = host(lat.spins).copy()
    lat.set_counters(start, 0)
    lat.sweep([beta], 3)
    oracle.ising_run(2, L, s, beta, seed, oracle.lattice_id(0, 0, 0), start, 3, series=False)
    assert np.array_equal(host(lat.spins), s)
    before = lat.spins.clone()
    with pytest.raises(B.SpinError):
        lat.sweep([beta], 2)
    assert torch.equal(lat.spins, before) and lat.sweeps_done == start + 3


def test_double_checkerboard_hundred_hits():
    """The paper's k = 100 (Sec. 3.4) on a small lattice, both orders."""
    L, T, k, seed = 32, 8, 100, 29
    for order in (B.SPIN_ORDER_DCB, B.SPIN_ORDER_DCB_SYMMETRIC):
        lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
        lat.set_update_order(order, T, k)
        lat.sweep([0.4407], 2 * k)
        lid = oracle.lattice_id(0, 0, 0)
        s = oracle.ising_init(2, L, seed, lid)
        oracle.dcb_sweeps(L, s, 0.4407, seed, lid, 0, 2 * k, T, k, order == B.SPIN_ORDER_DCB_SYMMETRIC)
        assert np.array_equal(host(lat.spins), s), order


def test_binding_checks_arrays_against_the_handle():
    """The ABI takes host betas and device buffers without lengths; the
    binding checks them against the handle's descriptor and refuses short,
    mistyped or host arrays before the call, leaving the handle unchanged."""
    lat = sp.Lattice(B.SPIN_ISING, 2, 32, B.SPIN_I8, n_temps=3, seed=41)
    before = lat.spins.clone()
    with pytest.raises(B.SpinError):
        lat.sweep([0.4, 0.5], 1)  # three slots
    short = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(B.SpinError):
        B.spin_measure(lat.h, None, E=short)
    with pytest.raises(B.SpinError):
        B.spin_measure(lat.h, None, E=torch.zeros(3, dtype=torch.int32, device="cuda"))
    with pytest.raises(B.SpinError):
        B.spin_measure(lat.h, None, M=torch.zeros(3, dtype=torch.int64))  # host tensor
    with pytest.raises(B.SpinError):  # 4 measurement rows need 12 entries
        B.spin_run(lat.h, None, [0.4, 0.5, 0.6], 8, 2, 0, torch.zeros(11, dtype=torch.int64, device="cuda"))
    with pytest.raises(B.SpinError):
        lat.pack(torch.ones(32 * 32, dtype=torch.int8, device="cuda"))  # one lattice of three
    assert torch.equal(lat.spins, before) and lat.sweeps_done == 0
    d = B.spin_describe(lat.h)
    assert (d.model, d.dim, d.L, d.layout, d.n_temps) == (B.SPIN_ISING, 2, 32, B.SPIN_I8, 3)
    ok = torch.zeros(12, dtype=torch.int64, device="cuda")
    B.spin_run(lat.h, None, [0.4, 0.5, 0.6], 8, 2, 0, ok)
    assert lat.sweeps_done == 8


def test_batched_launch_refuses_2d_coded_glass():
    """The batched launch takes 3D coded EA handles only; a 2D one is
    refused before anything runs."""
    ea = sp.Lattice(B.SPIN_EA, 2, 16, B.SPIN_MSC1, n_real=32, n_temps=2, n_sets=2, seed=3)
    before = ea.spins.clone()
    with pytest.raises(B.SpinError):
        sp.batch_run([ea.batch_item([0.5, 0.7])], 2, 0, 0)
    assert torch.equal(ea.spins, before) and ea.sweeps_done == 0


def test_variant_is_checked_against_the_handle():
    """Variant 3 (whole lattice in one CTA's shared memory) exists for int8
    ferromagnets with L % 8 == 0 and L <= 128 (2D) or L <= 24 (3D) only, and
    is their default; elsewhere it is refused."""
    small = sp.Lattice(B.SPIN_ISING, 2, 128, B.SPIN_I8, seed=3)
    small.set_variant(3)
    sp.Lattice(B.SPIN_ISING, 3, 24, B.SPIN_I8, seed=3).set_variant(3)
    for args in ((B.SPIN_ISING, 2, 256, B.SPIN_I8), (B.SPIN_ISING, 2, 20, B.SPIN_I8),
                 (B.SPIN_ISING, 2, 256, B.SPIN_MSC1), (B.SPIN_ISING, 3, 32, B.SPIN_I8),
                 (B.SPIN_ISING, 3, 12, B.SPIN_I8)):
        lat = sp.Lattice(*args, seed=3)
        with pytest.raises(B.SpinError):
            lat.set_variant(3)
    with pytest.raises(B.SpinError):
        small.set_variant(4)
