"""The allocation-free Heisenberg reduction (for callers that cannot allocate
device memory, e.g. inside a framework that owns the memory pool) must give
the same energies and magnetisations as the regular spin_measure, on two
calls in a row.  Kept in a file of its own that pytest collects last."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


def test_noalloc_reduction_matches_spin_measure_twice():
    L, n_temps = 16, 3
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, L, B.SPIN_F32X4, n_temps=n_temps, seed=21)
    betas = [0.3, 0.693, 1.2]
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-9 * L ** 3  # the tolerance of the Heisenberg reduction tests
    for _ in range(2):
        lat.sweep(betas, 7)
        Ef, Mf = lat.measure()
        Ef2 = torch.full((n_temps,), float("nan"), dtype=torch.float64, device="cuda")
        Mf2 = torch.full((3 * n_temps,), float("nan"), dtype=torch.float64, device="cuda")
        B.spin_heis_measure_noalloc(lat.spins, L, n_temps, Ef2, Mf2, stream)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(Ef - Ef2)).item() <= tol
        assert torch.max(torch.abs(Mf.view(-1) - Mf2)).item() <= tol


def test_noalloc_rejects_sizes_beyond_its_scratch():
    spins = torch.zeros(4 * 4 ** 3 * 2, dtype=torch.float32, device="cuda")
    with pytest.raises(B.SpinError) as e:
        B.spin_heis_measure_noalloc(spins, 4, 257)
    assert e.value.code == B.SPIN_EINVAL
