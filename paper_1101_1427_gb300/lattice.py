"""A library handle together with the device tensors it borrows.

PyTorch provides the device memory and the stream; the spins, couplings and
measurement buffers are plain CUDA tensors whose pointers are passed through
the C ABI.  No arithmetic of the method happens here.
"""
import torch

from . import _binding as B


def _words(model, layout, dim, L, n_real, n_temps, n_sets):
    N = L ** dim
    n_lat = n_sets * n_temps * n_real
    if layout == B.SPIN_I8:
        return torch.int8, n_lat * N
    if layout == B.SPIN_F32X4:
        return torch.float32, 4 * n_lat * N
    if model == B.SPIN_EA:
        return torch.int32, n_sets * (n_real // 32) * n_temps * N
    return torch.int32, n_lat * 2 * L * (L // 64)


class Lattice:
    """Spins (and couplings) on the current CUDA device plus a handle.

    model: SPIN_ISING / SPIN_EA / SPIN_HEISENBERG; layout: SPIN_I8 /
    SPIN_MSC1 / SPIN_F32X4.  Lattice index lat = (a * n_temps + t) * n_real + r.
    """

    def __init__(self, model, dim, L, layout, n_real=1, n_temps=1, n_sets=1, seed=1,
                 hot_start=True, stream=None, device=None):
        self.model, self.dim, self.L, self.layout = model, dim, L, layout
        self.n_real, self.n_temps, self.n_sets = n_real, n_temps, n_sets
        self.seed = seed
        self.N = L ** dim
        self.n_lat = n_sets * n_temps * n_real
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        dtype, count = _words(model, layout, dim, L, n_real, n_temps, n_sets)
        self.spins = torch.empty(count, dtype=dtype, device=self.device)
        self.couplings = None
        if model == B.SPIN_EA:
            if layout == B.SPIN_I8:
                self.couplings = torch.empty(n_real * dim * self.N, dtype=torch.int8,
                                             device=self.device)
            else:
                self.couplings = torch.empty((n_real // 32) * dim * self.N, dtype=torch.int32,
                                             device=self.device)
        self.desc = B.spin_desc(model, dim, L, layout, n_real, n_temps, n_sets, int(hot_start),
                                seed, self.stream.cuda_stream)
        self.h = B.spin_init(self.desc, self.spins, self.couplings)

    # -------------------------------------------------------------- the ABI calls
    def sweep(self, betas, n_sweeps=1):
        B.spin_sweep(self.h, self.couplings, list(betas), n_sweeps, self.seed)

    def measure(self):
        """Returns device tensors (E, M, Q) or (Ef, Mf) for Heisenberg."""
        if self.model == B.SPIN_HEISENBERG:
            Ef = torch.empty(self.n_lat, dtype=torch.float64, device=self.device)
            Mf = torch.empty(self.n_lat * 3, dtype=torch.float64, device=self.device)
            B.spin_measure(self.h, None, Ef=Ef, Mf=Mf)
            return Ef, Mf.view(self.n_lat, 3)
        E = torch.empty(self.n_lat, dtype=torch.int64, device=self.device)
        M = torch.empty(self.n_lat, dtype=torch.int64, device=self.device)
        Q = None
        if self.n_sets >= 2:
            Q = torch.empty(self.n_temps * self.n_real, dtype=torch.int64, device=self.device)
        B.spin_measure(self.h, self.couplings, E=E, M=M, Q=Q)
        return E, M, Q

    def pt_swap(self, betas, accepted=None, labels=None):
        B.spin_pt_swap(self.h, self.couplings, list(betas), self.seed, accepted, labels)

    def slot_labels(self):
        """Configuration labels [n_sets, n_temps, n_real] (int32, device)
        holding each lattice's slot t: passed to pt_swap / run / batch_item,
        they follow the configurations through accepted exchanges."""
        t = torch.arange(self.n_temps, dtype=torch.int32, device=self.device)
        return t.view(1, -1, 1).expand(self.n_sets, self.n_temps, self.n_real).contiguous()

    def run(self, betas, n_sweeps, measure_every=0, pt_every=0, series=True, accepted=None,
            labels=None):
        # measurements fall on sweep counts that are multiples of measure_every,
        # counted from the handle's counter (not from the start of the call)
        n_meas = B._n_meas(self.h, n_sweeps, measure_every)
        out = {}
        if series and n_meas:
            if self.model == B.SPIN_HEISENBERG:
                out["Ef"] = torch.empty(n_meas * self.n_lat, dtype=torch.float64, device=self.device)
                out["Mf"] = torch.empty(n_meas * self.n_lat * 3, dtype=torch.float64,
                                        device=self.device)
            else:
                out["E"] = torch.empty(n_meas * self.n_lat, dtype=torch.int64, device=self.device)
                out["M"] = torch.empty(n_meas * self.n_lat, dtype=torch.int64, device=self.device)
                if self.n_sets >= 2:
                    out["Q"] = torch.empty(n_meas * self.n_temps * self.n_real, dtype=torch.int64,
                                           device=self.device)
        B.spin_run(self.h, self.couplings, list(betas), n_sweeps, measure_every, pt_every,
                   out.get("E"), out.get("M"), out.get("Q"), out.get("Ef"), out.get("Mf"),
                   accepted, labels)
        return out

    def series_buffers(self, n_meas):
        """Device tensors for n_meas measurements (as filled by run / batch)."""
        out = {}
        if self.model == B.SPIN_HEISENBERG:
            return out
        out["E"] = torch.zeros(n_meas * self.n_lat, dtype=torch.int64, device=self.device)
        out["M"] = torch.zeros(n_meas * self.n_lat, dtype=torch.int64, device=self.device)
        if self.n_sets >= 2:
            out["Q"] = torch.zeros(n_meas * self.n_temps * self.n_real, dtype=torch.int64,
                                   device=self.device)
        return out

    def batch_item(self, betas, series=None, accepted=None, labels=None):
        it = {"lat": self.h, "couplings": self.couplings, "betas": list(betas)}
        if series:
            it.update(series)
        if accepted is not None:
            it["accepted"] = accepted
        if labels is not None:
            it["labels"] = labels
        return it

    def unpack(self):
        """Spins as int8 +-1, shape [n_sets, n_temps, n_real, N] (I8 / MSC1)."""
        out = torch.empty(self.n_lat * self.N, dtype=torch.int8, device=self.device)
        B.spin_unpack_i8(self.h, out)
        return out.view(self.n_sets, self.n_temps, self.n_real, self.N)

    def pack(self, spins_i8):
        B.spin_pack_i8(self.h, spins_i8.contiguous().view(-1))

    def sync(self):
        B.spin_sync(self.h)

    @property
    def sweeps_done(self):
        return B.spin_sweeps_done(self.h)

    @property
    def pt_steps_done(self):
        return B.spin_pt_steps_done(self.h)

    def set_counters(self, sweeps_done, pt_steps_done=0):
        B.spin_set_counters(self.h, sweeps_done, pt_steps_done)

    def set_variant(self, variant):
        B.spin_set_variant(self.h, variant)

    def set_msc_width(self, width):
        B.spin_set_msc_width(self.h, width)

    def tune(self, betas, n_sweeps):
        """Autotunes the kernel form (and an open double-checkerboard tile
        edge) for calls of n_sweeps sweeps; returns (variant, tile)."""
        return B.spin_tune(self.h, self.couplings, list(betas), n_sweeps)

    def set_update_order(self, order, tile=0, hits=1):
        B.spin_set_update_order(self.h, order, tile, hits)

    # -------------------------------------------------------------- checkpoints
    def state_dict(self):
        """Everything a chain needs to continue: the generator is counter
        based, so the state is the spins, the couplings, the seed and the
        two counters (the betas and the update order are the caller's)."""
        self.sync()
        return {"desc": [self.model, self.dim, self.L, self.layout, self.n_real, self.n_temps,
                         self.n_sets, self.seed],
                "spins": self.spins.detach().cpu().clone(),
                "couplings": None if self.couplings is None else self.couplings.detach().cpu().clone(),
                "sweeps_done": self.sweeps_done, "pt_steps_done": self.pt_steps_done}

    def save(self, path):
        torch.save(self.state_dict(), path)

    @classmethod
    def from_state_dict(cls, state, stream=None, device=None):
        model, dim, L, layout, n_real, n_temps, n_sets, seed = state["desc"]
        lat = cls(model, dim, L, layout, n_real=n_real, n_temps=n_temps, n_sets=n_sets, seed=seed,
                  stream=stream, device=device)
        lat.spins.copy_(state["spins"])
        if state["couplings"] is not None:
            lat.couplings.copy_(state["couplings"])
        lat.set_counters(state["sweeps_done"], state["pt_steps_done"])
        return lat

    @classmethod
    def load(cls, path, stream=None, device=None):
        return cls.from_state_dict(torch.load(path, weights_only=False), stream=stream, device=device)

    def close(self):
        if self.h is not None:
            B.spin_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_run(items, n_sweeps, measure_every=0, pt_every=0, stream=None):
    """One batched persistent launch over several lattices (see spin_batch_run)."""
    stream = stream or torch.cuda.current_stream()
    B.spin_batch_run(items, n_sweeps, measure_every, pt_every, stream.cuda_stream)


class BatchGraph:
    """One batched launch (see spin_batch_run) captured into a CUDA graph.

    Every ``replay()`` runs ``n_sweeps`` more sweeps of all handles, with the
    measurements and exchanges of the captured call, continuing each
    handle's random streams; the handles' host counters follow the replays.
    The series buffers named by the items are rewritten by every replay.
    """

    def __init__(self, items, n_sweeps, measure_every=0, pt_every=0):
        self.n_sweeps, self.pt_every = n_sweeps, pt_every
        self.handles = [it["lat"] for it in items]
        cur = torch.cuda.current_stream()
        # tables, workspace and device counters, outside the capture
        B.spin_batch_run(items, 0, measure_every, pt_every, cur.cuda_stream)
        before = [(B.spin_sweeps_done(h), B.spin_pt_steps_done(h)) for h in self.handles]
        side = torch.cuda.Stream()
        side.wait_stream(cur)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            B.spin_batch_run(items, n_sweeps, measure_every, pt_every, side.cuda_stream)
        cur.wait_stream(side)
        # the capture ran nothing: the counters stand where they were
        for h, (sw, pt) in zip(self.handles, before):
            B.spin_set_counters(h, sw, pt)

    def replay(self):
        self.graph.replay()
        for h in self.handles:
            sw, pt = B.spin_sweeps_done(h), B.spin_pt_steps_done(h)
            if self.pt_every > 0:
                pt += (sw + self.n_sweeps) // self.pt_every - sw // self.pt_every
            B.spin_set_counters(h, sw + self.n_sweeps, pt)

