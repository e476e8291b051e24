"""Named workloads: the five configurations this library is measured on,
each as the handles it needs (with their betas) and its run schedule.

    from paper_1101_1427_gb300 import presets
    p = presets.build("ea3d_L16_pt")          # handles on the current GPU
    out = presets.run(p, n_sweeps=100)         # series of E, M (and Q)

Temperatures T spaced geometrically in an interval use beta = 1 / T with
slot 0 at the lowest T; every lattice starts hot from its seed.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import _binding as B


@dataclass
class Member:
    """One handle of a preset: Lattice arguments and its betas."""
    model: int
    dim: int
    L: int
    layout: int
    betas: List[float]
    n_real: int = 1
    n_sets: int = 1
    seed: int = 1


@dataclass
class Preset:
    name: str
    members: List[Member]
    n_sweeps: int
    measure_every: int
    pt_every: int = 0
    batched: bool = False  # one persistent launch for all members
    lattices: list = field(default_factory=list)


def _geom_betas(t_lo, t_hi, n):
    return list(1.0 / np.geomspace(t_lo, t_hi, n))


UNEVEN_EA = [(8, 512, 24), (12, 256, 30), (16, 128, 36), (24, 64, 42), (32, 32, 48)]
UNEVEN_ISING = [256, 512, 1024, 2048, 4096]


def definitions():
    """The presets by name (no GPU work)."""
    uneven = [Member(B.SPIN_EA, 3, L, B.SPIN_MSC1, _geom_betas(0.8, 2.2, T), n_real=R, n_sets=2, seed=50 + k)
              for k, (L, R, T) in enumerate(UNEVEN_EA)]
    uneven += [Member(B.SPIN_ISING, 2, L, B.SPIN_MSC1, [0.4407], seed=60 + k) for k, L in enumerate(UNEVEN_ISING)]
    return {
        # 2D Ising L=64, int8, at the critical coupling; E and M every sweep
        "ising2d_L64": Preset("ising2d_L64", [Member(B.SPIN_ISING, 2, 64, B.SPIN_I8, [0.4407])], 1000, 1),
        # 2D Ising L=16384 (2^28 spins), three lattices, 1-bit coded (the int8
        # layout is the same preset with layout SPIN_I8)
        "ising2d_L16384": Preset("ising2d_L16384",
                                 [Member(B.SPIN_ISING, 2, 16384, B.SPIN_MSC1, [0.40, 0.4407, 0.50])], 1000, 10),
        # 3D Heisenberg L=128, FP32, renormalised every 100 sweeps by the library
        "heisenberg3d_L128": Preset("heisenberg3d_L128",
                                    [Member(B.SPIN_HEISENBERG, 3, 128, B.SPIN_F32X4, [0.693])], 2000, 100),
        # 3D +-J EA L=16: 1024 realisations x 32 temperatures in [0.9, 2.0] x 2
        # replica sets, coded; exchange and E, M, Q every sweep, batched
        "ea3d_L16_pt": Preset("ea3d_L16_pt",
                              [Member(B.SPIN_EA, 3, 16, B.SPIN_MSC1, _geom_betas(0.9, 2.0, 32), n_real=1024,
                                      n_sets=2)], 10000, 1, 1, batched=True),
        # EA L = 8..32 and 2D Ising L = 256..4096 in one persistent launch
        "uneven_batch": Preset("uneven_batch", uneven, 5000, 1, 1, batched=True),
    }


def build(name, device=None):
    """Creates the preset's handles (hot start) on the current CUDA device."""
    from .lattice import Lattice
    p = definitions()[name]
    # a member's temperature slots are its betas
    p.lattices = [Lattice(m.model, m.dim, m.L, m.layout, n_real=m.n_real, n_temps=len(m.betas),
                          n_sets=m.n_sets, seed=m.seed, device=device) for m in p.members]
    return p


def run(p, n_sweeps=None):
    """Runs a built preset for n_sweeps (default: its own count, which must
    then be a multiple of measure_every); returns one dict of device series
    per member (E, M, Q or Ef, Mf)."""
    from .lattice import batch_run
    n = p.n_sweeps if n_sweeps is None else n_sweeps
    if p.batched:
        outs = []
        items = []
        for lat, m in zip(p.lattices, p.members):
            # measurements fall on the handle's sweep counts that are multiples of measure_every
            ser = lat.series_buffers(B._n_meas(lat.h, n, p.measure_every))
            if lat.n_sets < 2:
                ser.pop("Q", None)
            outs.append(ser)
            items.append(lat.batch_item(m.betas, ser))
        has_pt = any(lat.model == B.SPIN_EA for lat in p.lattices)
        batch_run(items, n, p.measure_every, p.pt_every if has_pt else 0)
        return outs
    return [lat.run(m.betas, n, measure_every=p.measure_every,
                    pt_every=p.pt_every if lat.model == B.SPIN_EA else 0)
            for lat, m in zip(p.lattices, p.members)]
