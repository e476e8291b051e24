"""The named presets describe the five workloads as documented (no GPU),
and each one builds and runs a few sweeps on the GPU with its last
measurement equal to a fresh measurement of the final state."""
import numpy as np
import pytest

from paper_1101_1427_gb300 import _binding as B
from paper_1101_1427_gb300 import presets


def test_definitions_match_the_workloads():
    d = presets.definitions()
    assert set(d) == {"ising2d_L64", "ising2d_L16384", "heisenberg3d_L128", "ea3d_L16_pt", "uneven_batch"}
    assert d["ising2d_L64"].n_sweeps == 1000 and d["ising2d_L64"].measure_every == 1
    assert d["ising2d_L16384"].members[0].betas == [0.40, 0.4407, 0.50]
    assert d["heisenberg3d_L128"].n_sweeps == 2000
    ea = d["ea3d_L16_pt"].members[0]
    assert (ea.L, ea.n_real, len(ea.betas), ea.n_sets) == (16, 1024, 32, 2)
    assert np.isclose(ea.betas[0], 1 / 0.9) and np.isclose(ea.betas[-1], 1 / 2.0)
    assert d["ea3d_L16_pt"].n_sweeps == 10000 and d["ea3d_L16_pt"].pt_every == 1
    # spins per sweep of the uneven batch: 274,202,624
    u = d["uneven_batch"]
    spins = sum(m.L ** m.dim * m.n_real * len(m.betas) * m.n_sets for m in u.members)
    assert spins == 274_202_624 and u.n_sweeps == 5000 and u.batched
    assert [len(m.betas) for m in u.members if m.model == B.SPIN_EA] == [24, 30, 36, 42, 48]
    assert all(np.isclose(1 / m.betas[0], 0.8) and np.isclose(1 / m.betas[-1], 2.2)
               for m in u.members if m.model == B.SPIN_EA)


@pytest.mark.gpu
@pytest.mark.parametrize("name,n", [("ising2d_L64", 5), ("ising2d_L16384", 10), ("heisenberg3d_L128", 100),
                                    ("ea3d_L16_pt", 3), ("uneven_batch", 2)])
def test_presets_run(name, n):
    torch = pytest.importorskip("torch")
    p = presets.build(name)
    outs = presets.run(p, n)
    torch.cuda.synchronize()
    for lat, out in zip(p.lattices, outs):
        rows = n // p.measure_every
        if lat.model == B.SPIN_HEISENBERG:
            Ef, _ = lat.measure()
            last = out["Ef"].view(rows, lat.n_lat)[-1]
            assert torch.allclose(last, Ef, rtol=0, atol=1e-6 * lat.N)
        else:
            E, M, _ = lat.measure()
            last_E, last_M = out["E"].view(rows, lat.n_lat)[-1], out["M"].view(rows, lat.n_lat)[-1]
            if p.pt_every and lat.model == B.SPIN_EA:
                # the series is measured before the same sweep's exchange, which
                # permutes configurations among the slots of each (set, realisation)
                shape = (lat.n_sets, lat.n_temps, lat.n_real)
                srt = lambda x: torch.sort(x.view(shape), dim=1).values
                assert torch.equal(srt(last_E), srt(E)) and torch.equal(srt(last_M), srt(M))
            else:
                assert torch.equal(last_E, E) and torch.equal(last_M, M)
        assert lat.sweeps_done == n
