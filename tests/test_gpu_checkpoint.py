"""Checkpoint and resume: n sweeps, save, load into a fresh handle, n more
sweeps equals 2n uninterrupted sweeps bit for bit (the generator is counter
based, so spins + couplings + seed + counters are the whole state)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402


CASES = {
    "ising2d_i8": (B.SPIN_ISING, 2, 64, B.SPIN_I8, 1, 3, 1, [0.3, 0.44, 0.6], 0),
    "ising2d_msc": (B.SPIN_ISING, 2, 256, B.SPIN_MSC1, 1, 2, 1, [0.4, 0.5], 0),
    "ea3d_msc_pt": (B.SPIN_EA, 3, 8, B.SPIN_MSC1, 64, 6, 2, list(1.0 / np.geomspace(0.9, 2.0, 6)), 1),
    "ea3d_i8_pt": (B.SPIN_EA, 3, 6, B.SPIN_I8, 4, 4, 2, list(1.0 / np.geomspace(0.9, 2.0, 4)), 2),
    "heis": (B.SPIN_HEISENBERG, 3, 16, B.SPIN_F32X4, 1, 1, 1, [0.693], 0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_resume_equals_uninterrupted(name, tmp_path):
    model, dim, L, layout, R, T, S, betas, pt = CASES[name]
    n = 6
    whole = sp.Lattice(model, dim, L, layout, n_real=R, n_temps=T, n_sets=S, seed=33)
    whole.run(betas, 2 * n, 0, pt, series=False)
    first = sp.Lattice(model, dim, L, layout, n_real=R, n_temps=T, n_sets=S, seed=33)
    first.run(betas, n, 0, pt, series=False)
    path = tmp_path / "state.pt"
    first.save(path)
    first.close()
    resumed = sp.Lattice.load(path)
    resumed.run(betas, n, 0, pt, series=False)
    assert resumed.sweeps_done == whole.sweeps_done == 2 * n
    assert resumed.pt_steps_done == whole.pt_steps_done
    assert torch.equal(resumed.spins, whole.spins)


def test_resume_batched_graph_chain(tmp_path):
    """A checkpoint taken between graph replays of a batched launch resumes
    into plain calls that continue the same chain."""
    betas = list(1.0 / np.geomspace(0.8, 2.2, 6))
    make = lambda: sp.Lattice(B.SPIN_EA, 3, 8, B.SPIN_MSC1, n_real=64, n_temps=6, n_sets=2, seed=44)
    a, b = make(), make()
    g = sp.BatchGraph([a.batch_item(betas)], 4, 0, 1)
    g.replay()
    g.replay()
    a.save(tmp_path / "a.pt")
    c = sp.Lattice.load(tmp_path / "a.pt")
    c.run(betas, 4, 0, 1, series=False)
    b.run(betas, 12, 0, 1, series=False)
    assert torch.equal(c.spins, b.spins)
