"""The allocation-free Heisenberg reduction (for callers that cannot allocate
device memory, e.g. inside a framework that owns the memory pool) must give
the same energies and magnetisations as the regular spin_measure -- bit for
bit, since both use one device function in one summation order -- on two
calls in a row, and the FP64 oracle's values on an oracle-made state.  Kept
in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


@pytest.mark.parametrize("dim,L", [(3, 16), (2, 48)])
def test_noalloc_reduction_matches_spin_measure_twice(dim, L):
    n_temps = 3
    lat = sp.Lattice(B.SPIN_HEISENBERG, dim, L, B.SPIN_F32X4, n_temps=n_temps, seed=21)
    betas = [0.3, 0.693, 1.2]
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        lat.sweep(betas, 7)
        Ef, Mf = lat.measure()
        Ef2 = torch.full((n_temps,), float("nan"), dtype=torch.float64, device="cuda")
        Mf2 = torch.full((3 * n_temps,), float("nan"), dtype=torch.float64, device="cuda")
        B.spin_heis_measure_noalloc(lat.spins, dim, L, n_temps, Ef2, Mf2, stream)
        torch.cuda.synchronize()
        assert torch.equal(Ef, Ef2)
        assert torch.equal(Mf.view(-1), Mf2)
    lat.close()


@pytest.mark.parametrize("dim,L", [(3, 12), (2, 40)])
def test_noalloc_reduction_matches_oracle(dim, L):
    """States from the oracle's Heisenberg hot start, rounded to FP32: the
    sums agree with the oracle's FP64 energy and magnetisation of the same
    FP32 values up to the rounding of a different summation order."""
    n_lat = 4
    N = L ** dim
    host = np.zeros((n_lat, N, 4), np.float32)
    E_or, M_or = [], []
    for k in range(n_lat):
        s = oracle.heis_init(dim, L, 30 + k, oracle.lattice_id(0, k, 0)).astype(np.float32)
        host[k, :, :3] = s
        sd = s.astype(np.float64)
        E_or.append(oracle.heis_energy(dim, L, sd))
        M_or.append(oracle.heis_magnetisation(dim, L, sd))
    spins = torch.from_numpy(host.reshape(-1)).cuda()
    Ef = torch.empty(n_lat, dtype=torch.float64, device="cuda")
    Mf = torch.empty(3 * n_lat, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        B.spin_heis_measure_noalloc(spins, dim, L, n_lat, Ef, Mf, stream)
        torch.cuda.synchronize()
        tol = 1e-12 * N  # FP32 products are exact in double; only the order differs
        assert np.max(np.abs(Ef.cpu().numpy() - np.array(E_or))) <= tol
        assert np.max(np.abs(Mf.cpu().numpy().reshape(n_lat, 3) - np.array(M_or))) <= tol


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """The library itself (called through ctypes, past the binding's own
    size checks) refuses requests its fixed array cannot hold and bad shapes."""
    lib = B.lib()
    spins = torch.zeros(4 * 257 * 4 ** 3, dtype=torch.float32, device="cuda")
    Ef = torch.zeros(257, dtype=torch.float64, device="cuda")
    p = C.c_void_p(spins.data_ptr())
    e = C.c_void_p(Ef.data_ptr())
    assert lib.spin_heis_measure_noalloc(p, 3, 4, 257, e, None, None) == B.SPIN_EINVAL
    assert lib.spin_heis_measure_noalloc(p, 4, 4, 1, e, None, None) == B.SPIN_EINVAL
    assert lib.spin_heis_measure_noalloc(p, 3, 1292, 1, e, None, None) == B.SPIN_EINVAL
    assert lib.spin_heis_measure_noalloc(p, 3, 5, 1, e, None, None) == B.SPIN_EINVAL
    # the largest request the array holds is accepted
    assert lib.spin_heis_measure_noalloc(p, 3, 4, 256, e, None, None) == B.SPIN_OK
    torch.cuda.synchronize()
