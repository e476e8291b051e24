"""Out-of-bounds writes: every device buffer handed to the library (spins,
couplings, series, exchange counters) sits between two guard bands of a
known byte pattern; after sweeps, measurements, exchange steps and batched
launches in every model, layout and update order the guard bands must be
untouched (a check for stray writes that needs no sanitizer)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1101_1427_gb300 import _binding as B  # noqa: E402
from paper_1101_1427_gb300.lattice import _words  # noqa: E402

PAD = 4096  # bytes on each side (keeps 16-byte alignment)
PATTERN = 0x5A


class Guarded:
    """A device buffer of n elements of dtype between two guard bands."""

    def __init__(self, n, dtype, fill=None):
        esz = torch.tensor([], dtype=dtype).element_size()
        self.raw = torch.full((2 * PAD + n * esz,), PATTERN, dtype=torch.uint8, device="cuda")
        self.t = self.raw[PAD:PAD + n * esz].view(dtype)
        if fill is not None:
            self.t.fill_(fill)

    def intact(self):
        torch.cuda.synchronize()
        return bool((self.raw[:PAD] == PATTERN).all()) and bool((self.raw[-PAD:] == PATTERN).all())


class Handle:
    def __init__(self, model, dim, L, layout, n_real=1, n_temps=1, n_sets=1, seed=3):
        self.model, self.dim, self.L, self.layout = model, dim, L, layout
        self.n_real, self.n_temps, self.n_sets = n_real, n_temps, n_sets
        self.n_lat = n_real * n_temps * n_sets
        self.seed = seed
        dtype, count = _words(model, layout, dim, L, n_real, n_temps, n_sets)
        self.spins = Guarded(count, dtype)
        self.J = None
        if model == B.SPIN_EA:
            N = L ** dim
            self.J = (Guarded(n_real * dim * N, torch.int8) if layout == B.SPIN_I8
                      else Guarded((n_real // 32) * dim * N, torch.int32))
        st = torch.cuda.current_stream()
        desc = B.spin_desc(model, dim, L, layout, n_real, n_temps, n_sets, 1, seed, st.cuda_stream)
        self.h = B.spin_init(desc, self.spins.t, self.J.t if self.J else None)
        self.guards = [self.spins] + ([self.J] if self.J else [])

    @property
    def couplings(self):
        return self.J.t if self.J else None

    def series(self, rows):
        heis = self.model == B.SPIN_HEISENBERG
        out = {}
        if heis:
            out["Ef"] = Guarded(rows * self.n_lat, torch.float64, 0)
            out["Mf"] = Guarded(3 * rows * self.n_lat, torch.float64, 0)
        else:
            out["E"] = Guarded(rows * self.n_lat, torch.int64, 0)
            out["M"] = Guarded(rows * self.n_lat, torch.int64, 0)
            if self.n_sets >= 2:
                out["Q"] = Guarded(rows * self.n_temps * self.n_real, torch.int64, 0)
        self.guards += list(out.values())
        return out

    def accepted(self):
        g = Guarded(self.n_sets * self.n_temps, torch.int64, 0)
        self.guards.append(g)
        return g

    def labels(self):
        g = Guarded(self.n_lat, torch.int32, 0)
        self.guards.append(g)
        return g

    def close(self):
        B.spin_destroy(self.h)


def _run_all(hd, betas, order=None):
    n = 4 if order is None else 2 * order[2]
    if order is not None:
        B.spin_set_update_order(hd.h, *order)
    ser = hd.series(n)
    pt = 1 if hd.model == B.SPIN_EA else 0
    acc = hd.accepted() if pt else None
    lab = hd.labels() if pt else None
    t = lambda k: ser[k].t if k in ser else None
    B.spin_run(hd.h, hd.couplings, betas, n, 1 if order is None else order[2], pt, t("E"), t("M"), t("Q"),
               t("Ef"), t("Mf"), acc.t if acc else None, lab.t if lab else None)
    one = hd.series(1)
    u = lambda k: one[k].t if k in one else None
    B.spin_measure(hd.h, hd.couplings, u("E"), u("M"), u("Q"), u("Ef"), u("Mf"))
    if pt:
        B.spin_pt_swap(hd.h, hd.couplings, betas, hd.seed, acc.t, lab.t)
    if hd.model != B.SPIN_HEISENBERG:
        out = Guarded(hd.n_lat * hd.L ** hd.dim, torch.int8)
        hd.guards.append(out)
        B.spin_unpack_i8(hd.h, out.t)
        B.spin_pack_i8(hd.h, out.t)
    B.spin_sync(hd.h)
    bad = [k for k, g in enumerate(hd.guards) if not g.intact()]
    assert not bad, f"guard bands overwritten in buffers {bad}"


CASES = [
    ("ising2d_i8_phases", (B.SPIN_ISING, 2, 40, B.SPIN_I8), dict(n_temps=3), 0, None),
    ("ising2d_i8_fused", (B.SPIN_ISING, 2, 48, B.SPIN_I8), dict(n_temps=2), 1, None),
    ("ising2d_i8_resident", (B.SPIN_ISING, 2, 40, B.SPIN_I8), dict(n_temps=3, n_real=2), 3, None),
    ("ising2d_i8_generic", (B.SPIN_ISING, 2, 6, B.SPIN_I8), dict(n_temps=2, n_real=2), 0, None),
    ("ising2d_coded", (B.SPIN_ISING, 2, 256, B.SPIN_MSC1), dict(n_temps=2), None, None),
    ("ising3d_i8_chunks", (B.SPIN_ISING, 3, 24, B.SPIN_I8), dict(n_temps=2), 0, None),
    ("ising3d_i8_resident", (B.SPIN_ISING, 3, 16, B.SPIN_I8), dict(n_temps=2, n_real=2), 3, None),
    ("ising3d_i8_generic", (B.SPIN_ISING, 3, 6, B.SPIN_I8), dict(n_temps=3), None, None),
    ("ising2d_dcb", (B.SPIN_ISING, 2, 64, B.SPIN_I8), dict(n_temps=2), None, (B.SPIN_ORDER_DCB_SYMMETRIC, 16, 2)),
    ("ising3d_dcb8", (B.SPIN_ISING, 3, 32, B.SPIN_I8), dict(n_temps=2), None, (B.SPIN_ORDER_DCB, 8, 2)),
    ("ising3d_dcb16", (B.SPIN_ISING, 3, 32, B.SPIN_I8), dict(), None, (B.SPIN_ORDER_DCB_SYMMETRIC, 16, 1)),
    ("ea3d_i8", (B.SPIN_EA, 3, 6, B.SPIN_I8), dict(n_real=3, n_temps=4, n_sets=2), None, None),
    ("ea3d_coded", (B.SPIN_EA, 3, 8, B.SPIN_MSC1), dict(n_real=64, n_temps=5, n_sets=2), None, None),
    ("ea2d_coded", (B.SPIN_EA, 2, 16, B.SPIN_MSC1), dict(n_real=64, n_temps=3, n_sets=2), None, None),
    ("ea2d_coded_persite", (B.SPIN_EA, 2, 10, B.SPIN_MSC1), dict(n_real=32, n_temps=2, n_sets=2), None, None),
    ("i8_2d_coded_path", (B.SPIN_ISING, 2, 256, B.SPIN_I8), dict(n_real=2), 4, None),
    ("heis3d", (B.SPIN_HEISENBERG, 3, 8, B.SPIN_F32X4), dict(n_temps=2), 2, None),
    ("heis2d", (B.SPIN_HEISENBERG, 2, 18, B.SPIN_F32X4), dict(n_temps=2), 0, None),
    ("heis2d_dcb8", (B.SPIN_HEISENBERG, 2, 32, B.SPIN_F32X4), dict(n_temps=2), 2, (B.SPIN_ORDER_DCB, 8, 2)),
    ("heis2d_dcb32", (B.SPIN_HEISENBERG, 2, 64, B.SPIN_F32X4), dict(), 0, (B.SPIN_ORDER_DCB_SYMMETRIC, 32, 1)),
]


@pytest.mark.parametrize("name,args,kw,variant,order", CASES, ids=[c[0] for c in CASES])
def test_no_stray_writes(name, args, kw, variant, order):
    hd = Handle(*args, **kw)
    if variant is not None:
        B.spin_set_variant(hd.h, variant)
    betas = list(np.linspace(0.3, 0.9, hd.n_temps))
    _run_all(hd, betas, order)
    hd.close()


@pytest.mark.parametrize("variant", [0, 2])
def test_no_stray_writes_heis3d_resident(variant):
    """3D Heisenberg L = 64 with two slots: calls of 6 sweeps and a run
    measuring every 4 sweeps take the resident kernel (pencils of two
    lattices in shared memory, faces through the handle's buffer)."""
    hd = Handle(B.SPIN_HEISENBERG, 3, 64, B.SPIN_F32X4, n_temps=2, seed=9)
    B.spin_set_variant(hd.h, variant)
    betas = [0.5, 0.9]
    B.spin_sweep(hd.h, None, betas, 6, hd.seed)
    ser = hd.series(2)
    B.spin_run(hd.h, None, betas, 8, 4, 0, None, None, None, ser["Ef"].t, ser["Mf"].t, None, None)
    _run_all(hd, betas)
    hd.close()


def test_no_stray_writes_w64_and_batch():
    ea = Handle(B.SPIN_EA, 3, 8, B.SPIN_MSC1, n_real=128, n_temps=4, n_sets=2, seed=5)
    B.spin_set_msc_width(ea.h, 64)
    _run_all(ea, [0.5, 0.7, 0.9, 1.1])
    B.spin_set_msc_width(ea.h, 32)
    ising = Handle(B.SPIN_ISING, 2, 256, B.SPIN_MSC1, seed=6)
    i8 = Handle(B.SPIN_ISING, 2, 32, B.SPIN_I8, seed=7)
    items, n = [], 3
    for hd, betas in ((ea, [0.5, 0.7, 0.9, 1.1]), (ising, [0.44]), (i8, [0.44])):
        ser = hd.series(n)
        acc = hd.accepted()
        lab = hd.labels()
        items.append({"lat": hd.h, "couplings": hd.couplings, "betas": betas,
                      **{k: g.t for k, g in ser.items()}, "accepted": acc.t, "labels": lab.t})
    B.spin_batch_run(items, n, 1, 1, torch.cuda.current_stream().cuda_stream)
    for hd in (ea, ising, i8):
        B.spin_sync(hd.h)
        bad = [k for k, g in enumerate(hd.guards) if not g.intact()]
        assert not bad, bad
        hd.close()


def test_guard_detects_a_modified_band():
    g = Guarded(100, torch.int32, 0)
    assert g.intact()
    g.raw[PAD - 1] = 0  # the byte just before the buffer
    assert not g.intact()
    g = Guarded(100, torch.int32, 0)
    g.raw[PAD + 400] = 0  # the byte just after it
    assert not g.intact()
