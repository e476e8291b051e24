"""Batched persistent launch (one cooperative kernel for many lattices and
many sweeps with fused measurement and exchange) against the per-handle
multi-launch path, which is itself bit-exact with the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1101_1427_gb300 as sp  # noqa: E402
from paper_1101_1427_gb300 import _binding as B  # noqa: E402

import oracle  # noqa: E402


def _make(kind, seed):
    if kind == "ea8":
        lat = sp.Lattice(B.SPIN_EA, 3, 8, B.SPIN_MSC1, n_real=64, n_temps=6, n_sets=2, seed=seed)
        betas = list(1.0 / np.geomspace(0.8, 2.2, 6))
    elif kind == "ea6":
        lat = sp.Lattice(B.SPIN_EA, 3, 6, B.SPIN_MSC1, n_real=32, n_temps=5, n_sets=2, seed=seed)
        betas = list(1.0 / np.geomspace(0.9, 2.0, 5))
    elif kind == "ising64":
        lat = sp.Lattice(B.SPIN_ISING, 2, 64, B.SPIN_I8, seed=seed)
        betas = [0.4407]
    elif kind == "ising96x2":
        lat = sp.Lattice(B.SPIN_ISING, 2, 96, B.SPIN_I8, n_temps=2, seed=seed)
        betas = [0.35, 0.5]
    elif kind == "coded512x2":
        lat = sp.Lattice(B.SPIN_ISING, 2, 512, B.SPIN_MSC1, n_temps=2, seed=seed)
        betas = [0.4, 0.5]
    return lat, betas


KINDS = ["ea8", "ea6", "ising64", "ising96x2", "coded512x2"]


@pytest.mark.parametrize("measure_every,pt_every", [(1, 1), (3, 2), (0, 1), (2, 0)])
def test_batch_equals_per_handle_runs(measure_every, pt_every):
    n = 12
    plain, batch = [], []
    for k, kind in enumerate(KINDS):
        plain.append(_make(kind, 100 + k))
        batch.append(_make(kind, 100 + k))
    n_meas = n // measure_every if measure_every else 0
    items, outs_b = [], []
    for (lat, betas) in batch:
        ser = lat.series_buffers(n_meas) if n_meas else {}
        if lat.n_sets < 2:
            ser.pop("Q", None)
        acc = torch.zeros(lat.n_sets * lat.n_temps, dtype=torch.int64, device="cuda")
        labels = lat.slot_labels() if lat.model == B.SPIN_EA else None
        items.append(lat.batch_item(betas, ser, acc, labels))
        outs_b.append((ser, acc, labels))
    ising_pt = pt_every and any(l.model == B.SPIN_ISING and l.n_temps > 1 for l, _ in batch)
    if ising_pt:
        with pytest.raises(B.SpinError):
            sp.batch_run(items, n, measure_every, pt_every)
        items = [it for it, (l, _) in zip(items, batch) if not (l.model == B.SPIN_ISING and l.n_temps > 1)]
        keep = [i for i, (l, _) in enumerate(batch) if not (l.model == B.SPIN_ISING and l.n_temps > 1)]
    else:
        keep = list(range(len(batch)))
    sp.batch_run(items, n, measure_every, pt_every)
    batch[0][0].sync()
    for i in keep:
        lat, betas = plain[i]
        acc = torch.zeros(lat.n_sets * lat.n_temps, dtype=torch.int64, device="cuda")
        labels = lat.slot_labels() if lat.model == B.SPIN_EA else None
        out = lat.run(betas, n, measure_every, pt_every if lat.model == B.SPIN_EA or lat.n_temps == 1 else 0,
                      accepted=acc, labels=labels)
        lb = batch[i][0]
        assert torch.equal(lat.spins, lb.spins), KINDS[i]
        ser, accb, labels_b = outs_b[i]
        if labels is not None:
            assert torch.equal(labels, labels_b), KINDS[i]
        for key in ("E", "M", "Q"):
            if key in out and key in ser:
                assert torch.equal(out[key], ser[key]), (KINDS[i], key)
        if lat.model == B.SPIN_EA:
            assert torch.equal(acc, accb), KINDS[i]
        assert lb.sweeps_done == lat.sweeps_done == n
        assert lb.pt_steps_done == lat.pt_steps_done


def test_batch_matches_oracle_for_one_realisation():
    L, seed, n = 6, 7, 8
    lat = sp.Lattice(B.SPIN_EA, 3, L, B.SPIN_MSC1, n_real=32, n_temps=4, n_sets=2, seed=seed)
    betas = list(1.0 / np.geomspace(0.9, 2.0, 4))
    ser = lat.series_buffers(n)
    labels = lat.slot_labels()
    sp.batch_run([lat.batch_item(betas, ser, labels=labels)], n, 1, 1)
    got = lat.unpack().cpu().numpy()
    E = ser["E"].cpu().numpy().reshape(n, 2, 4, 32)
    lab_gpu = labels.cpu().numpy()
    for r in (0, 17, 31):
        J = oracle.ea_couplings(3, L, r, seed)
        s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(a, 0, t), bit=r)
                                for t in range(4)]) for a in range(2)]).copy()
        lab = np.tile(np.arange(4, dtype=np.int32), (2, 1))
        Es, Qs, acc, _ = oracle.pt_run(3, L, s, betas, seed, r, 0, 0, n, 1, J=J, labels=lab)
        assert np.array_equal(got[:, :, r], s)
        assert np.array_equal(E[:, :, :, r], Es)
        assert np.array_equal(lab_gpu[:, :, r], lab)


def test_batch_timeout_is_reported_and_context_survives():
    lat, betas = _make("ea6", 3)
    B.spin_set_batch_options(lat.h, timeout_ns=50_000_000, missing_arrivals=1)
    sp.batch_run([lat.batch_item(betas)], 4, 0, 1)
    with pytest.raises(B.SpinError) as e:
        lat.sync()
    assert e.value.code == B.SPIN_ETIMEOUT
    B.spin_set_batch_options(lat.h)
    # the context is still usable
    other, ob = _make("ising64", 5)
    other.sweep(ob, 3)
    other.sync()


def test_batch_autotuner_keeps_state():
    items_l = [_make("ea8", 1), _make("ising64", 2)]
    before = [l.spins.clone() for l, _ in items_l]
    best = B.spin_batch_tune([l.batch_item(b) for l, b in items_l], 4, 0, 1,
                             torch.cuda.current_stream().cuda_stream)
    assert 1 <= best <= 4
    for (l, _), b in zip(items_l, before):
        assert torch.equal(l.spins, b) and l.sweeps_done == 0


def test_batch_graph_replays_continue_the_chain():
    """A batched launch captured into a CUDA graph: each replay equals the
    next uncaptured call on a twin set of handles (lattices, series,
    exchange counts, counters), and plain calls continue correctly after."""
    kinds = ["ea8", "ea6", "ising64"]
    n, me, pe = 4, 2, 1
    graph_side = [_make(k, 300 + i) for i, k in enumerate(kinds)]
    plain_side = [_make(k, 300 + i) for i, k in enumerate(kinds)]

    def items_for(side):
        items, outs = [], []
        for lat, betas in side:
            ser = lat.series_buffers(n // me)
            if lat.n_sets < 2:
                ser.pop("Q", None)
            acc = torch.zeros(lat.n_sets * lat.n_temps, dtype=torch.int64, device="cuda")
            items.append(lat.batch_item(betas, ser, acc))
            outs.append((ser, acc))
        return items, outs

    items_g, outs_g = items_for(graph_side)
    items_p, outs_p = items_for(plain_side)
    g = sp.BatchGraph(items_g, n, me, pe)
    for rep in range(3):
        g.replay()
        sp.batch_run(items_p, n, me, pe)
        torch.cuda.synchronize()
        for (lg, _), (lp, _), (sg, ag), (sp_, ap) in zip(graph_side, plain_side, outs_g, outs_p):
            assert torch.equal(lg.spins, lp.spins), rep
            for key in sg:
                assert torch.equal(sg[key], sp_[key]), (rep, key)
            assert torch.equal(ag, ap), rep
            assert lg.sweeps_done == lp.sweeps_done == n * (rep + 1)
            assert lg.pt_steps_done == lp.pt_steps_done
    graph_side[0][0].sync()
    for (lg, betas), (lp, _) in zip(graph_side, plain_side):
        pt = pe if lg.model == B.SPIN_EA else 0
        lg.run(betas, 3, 0, pt, series=False)
        lp.run(betas, 3, 0, pt, series=False)
        assert torch.equal(lg.spins, lp.spins)


def test_batch_w64_equals_plain_w64():
    """The batched launch keys the uniforms of a w = 64 handle by group pair,
    as the per-handle pair kernel does."""
    betas = list(1.0 / np.geomspace(0.8, 2.2, 5))
    make = lambda: sp.Lattice(B.SPIN_EA, 3, 8, B.SPIN_MSC1, n_real=128, n_temps=5, n_sets=2, seed=71)
    a, b = make(), make()
    a.set_msc_width(64)
    b.set_msc_width(64)
    ser = a.series_buffers(6)
    sp.batch_run([a.batch_item(betas, ser)], 6, 1, 1)
    out = b.run(betas, 6, 1, 1)
    a.sync()
    assert torch.equal(a.spins, b.spins)
    for key in ("E", "M", "Q"):
        assert torch.equal(ser[key], out[key]), key

