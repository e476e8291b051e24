"""Slab decomposition on the GPU (one GPU standing in for P ranks: P slab
buffers, ghost rows copied between them before every colour phase): the
gathered lattice equals the unsplit int8 sweep bit for bit, and the partial
E, M add up to the full measurement."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402
from paper_1101_1427_gb300 import slab as S  # noqa: E402


@pytest.mark.parametrize("L,P", [(256, 1), (256, 2), (264, 3), (1024, 4)])
def test_slabs_equal_unsplit_lattice(L, P):
    beta, seed, n = 0.4407, 19, 4
    full = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, seed=seed)
    start = full.spins.view(L, L).clone()
    full.sweep([beta], n)
    parts = [S.split_rows(L, P, k) for k in range(P)]
    slabs = []
    for y0, rows in parts:
        sl = torch.zeros(rows + 2, L, dtype=torch.int8, device="cuda")
        sl[1:rows + 1] = start[y0:y0 + rows]
        slabs.append(sl)
    for sweep in range(n):
        for colour in (0, 1):
            S.exchange_ghosts_local(slabs)
            for (y0, rows), sl in zip(parts, slabs):
                S.phase(sl, L, y0, rows, beta, seed, 0, sweep, colour)
    got = torch.cat([sl[1:-1] for sl in slabs])
    assert torch.equal(got, full.spins.view(L, L))
    S.exchange_ghosts_local(slabs)
    E = torch.zeros(P, dtype=torch.int64, device="cuda")
    M = torch.zeros(P, dtype=torch.int64, device="cuda")
    for k, ((_, rows), sl) in enumerate(zip(parts, slabs)):
        S.measure(sl, L, rows, E[k:k + 1], M[k:k + 1])
    Ef, Mf, _ = full.measure()
    assert E.sum().item() == Ef.item() and M.sum().item() == Mf.item()


def test_slab_rejects_bad_arguments():
    sl = torch.zeros(6, 64, dtype=torch.int8, device="cuda")
    for args in ((64, 0, 0), (60, 0, 4), (64, 62, 4), (64, -1, 4)):  # rows 0, L % 8, past the end, y0 < 0
        L, y0, rows = args
        with pytest.raises(B.SpinError):
            S.phase(sl, L, y0, rows, 0.4, 1, 0, 0, 0)
    with pytest.raises(B.SpinError):
        S.phase(sl, 64, 0, 4, 0.4, 1, 0, 0, 2)
