"""3D Heisenberg calls of at least 4 sweeps on lattices of L = 64 or 128
run resident in the SMs' shared memory (one pencil of rows per CTA, faces
exchanged with the four neighbour pencils through a global buffer, bounded
waits on per-CTA phase counters); shorter calls run one launch per colour
phase.  The per-site arithmetic is shared, so a chain is the same bit for
bit however its sweeps are split into calls: across a renormalisation
(every 100th sweep), in both variants, for one lattice of L = 128 and for
several lattices and temperature slots of L = 64.  Against the FP64 oracle
the resident path stays within the one-sweep tolerance outside near-ties,
and a neighbour wait that can never be satisfied ends in SPIN_ETIMEOUT with
the context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


def _pair(L, n_real, n_temps, variant, seed, start=94, n_sets=1):
    out = []
    for _ in range(2):
        lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, n_real=n_real, n_temps=n_temps, n_sets=n_sets,
                         seed=seed)
        lat.set_variant(variant)
        lat.set_counters(start, 0)  # the calls below cross the renormalisation after sweep 100
        out.append(lat)
    return out


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("L,n_real,n_temps,n_sets", [(128, 1, 1, 1), (64, 1, 3, 1), (64, 2, 2, 1), (64, 1, 2, 2)])
def test_resident_and_per_phase_kernels_give_one_chain(variant, L, n_real, n_temps, n_sets):
    betas = list(np.linspace(0.5, 1.1, n_temps))
    a, b = _pair(L, n_real, n_temps, variant, seed=43, n_sets=n_sets)
    for _ in range(12):
        a.sweep(betas, 1)  # one launch per colour phase
    b.sweep(betas, 12)  # resident: sweeps 94..99, renormalisation, 100..105
    assert a.sweeps_done == b.sweeps_done == 106
    assert torch.equal(a.spins, b.spins)
    b.sweep(betas, 5)
    for _ in range(5):
        a.sweep(betas, 1)
    assert torch.equal(a.spins, b.spins)
    b.sync()
    a.close()
    b.close()


@pytest.mark.parametrize("variant", [0, 2])
def test_resident_L128_chain_equals_colour_split_and_long_calls(variant):
    """Sweeps 0..203 of L = 128 in one call (two renormalisations inside),
    against calls of 3 sweeps (per-phase kernels)."""
    a, b = _pair(128, 1, 1, variant, seed=44, start=0)
    b.sweep([0.693], 204)
    for _ in range(68):
        a.sweep([0.693], 3)
    assert torch.equal(a.spins, b.spins)
    v = b.spins.view(-1, 4)[:, :3].double()
    assert torch.max(torch.abs(torch.linalg.norm(v, dim=1) - 1)).item() <= 1e-5
    a.close()
    b.close()


@pytest.mark.parametrize("variant", [0, 2])
def test_resident_four_sweeps_within_tolerance_of_fp64_oracle(variant):
    """Four sweeps in one resident call from an oracle state at high
    temperature: every component within 1e-5 of the FP64 oracle outside
    flagged near-ties (and the neighbourhoods they spread to)."""
    L, seed, beta, n = 64, 6, 0.3, 4
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, seed=seed)
    lat.set_variant(variant)
    s0 = oracle.heis_init(3, L, seed, 0).astype(np.float32)
    dev = np.zeros((L ** 3, 4), np.float32)
    dev[:, :3] = s0
    lat.spins.copy_(torch.from_numpy(dev.ravel()))
    lat.sweep([beta], n)
    got = lat.spins.view(-1, 4)[:, :3].cpu().numpy()
    ref = s0.astype(np.float64)
    margins = [oracle.heis_sweep(3, L, ref, beta, seed, 0, k, want_margin=True) for k in range(n)]
    flagged = np.min(np.stack(margins), axis=0) < 1e-5
    err = np.max(np.abs(got - ref), axis=1)
    assert (err > 1e-5).sum() <= 60 * max(1, int(flagged.sum()))
    if not flagged.any():
        assert err.max() <= 1e-5
    lat.close()


def test_resident_wait_timeout_is_reported_and_context_survives():
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, 64, B.SPIN_F32X4, seed=45)
    before = lat.spins.clone()
    B.spin_set_batch_options(lat.h, timeout_ns=20_000_000, missing_arrivals=1)
    lat.sweep([0.7], 6)
    with pytest.raises(B.SpinError) as e:
        lat.sync()
    assert e.value.code == B.SPIN_ETIMEOUT
    assert torch.equal(lat.spins, before)  # the launch ended before writing its pencils back
    B.spin_set_batch_options(lat.h)
    lat.sweep([0.7], 6)
    lat.sync()
    other = sp.Lattice(B.SPIN_HEISENBERG, 3, 64, B.SPIN_F32X4, seed=46)
    other.sweep([0.7], 5)
    other.sync()
    lat.close()
    other.close()


@pytest.mark.parametrize("variant", [0, 2])
def test_captured_sweeps_take_the_per_phase_kernels(variant):
    """Inside a stream capture the sweeps go through the per-phase kernels
    (nothing allocated, no published-phase counters to be met again by a
    later replay): one replay equals the same sweeps run resident."""
    s = torch.cuda.Stream()
    a = sp.Lattice(B.SPIN_HEISENBERG, 3, 64, B.SPIN_F32X4, seed=47, stream=s)
    b = sp.Lattice(B.SPIN_HEISENBERG, 3, 64, B.SPIN_F32X4, seed=47)
    for lat in (a, b):
        lat.set_variant(variant)
        lat.sweep([0.7], 1)  # uploads the thresholds outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.spin_sweep(a.h, None, [0.7], 6, a.seed)
    g.replay()
    torch.cuda.synchronize()
    b.sweep([0.7], 6)  # resident
    b.sync()
    assert a.sweeps_done == b.sweeps_done == 7
    assert torch.equal(a.spins, b.spins)
    a.close()
    b.close()


@pytest.mark.parametrize("variant", [0, 2])
def test_lattices_that_do_not_fit_take_the_other_paths(variant):
    """Two lattices of L = 128 (64 MiB) exceed the SMs' shared memory: long
    calls take the colour-split copy (fast math) or the per-phase kernel,
    with the same chain as calls of one sweep."""
    a, b = _pair(128, 1, 2, variant, seed=48, start=0)
    betas = [0.6, 0.9]
    b.sweep(betas, 5)
    for _ in range(5):
        a.sweep(betas, 1)
    assert torch.equal(a.spins, b.spins)
    a.close()
    b.close()
