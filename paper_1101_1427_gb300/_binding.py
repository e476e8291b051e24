"""Thin ctypes binding of the C ABI in include/spin.h.

Argument marshalling only: every step of the sweep, exchange and reduction
runs in the CUDA kernels of libspin_gb300.so.  There is no CPU fallback: if
the library is missing or no GPU is present the calls raise.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspin_gb300.so")

SPIN_OK, SPIN_EINVAL, SPIN_EALIGN, SPIN_ENOMEM, SPIN_ECUDA, SPIN_ETIMEOUT = 0, -1, -2, -3, -4, -5
SPIN_ISING, SPIN_EA, SPIN_HEISENBERG = 0, 1, 2
SPIN_I8, SPIN_MSC1, SPIN_F32X4 = 0, 1, 2
SPIN_ORDER_CHECKERBOARD, SPIN_ORDER_DCB, SPIN_ORDER_DCB_SYMMETRIC = 0, 1, 2
(SPIN_PIPE_MUL_WIDE, SPIN_PIPE_MAD_HI, SPIN_PIPE_LOP3, SPIN_PIPE_IADD3, SPIN_PIPE_FFMA,
 SPIN_PIPE_MUFU_RSQ) = range(6)
TAG_UPDATE, TAG_INIT, TAG_COUPLING, TAG_PT, TAG_HEIS, TAG_HEIS_INIT = range(6)


class spin_desc(C.Structure):
    _fields_ = [("model", C.c_int32), ("dim", C.c_int32), ("L", C.c_int32),
                ("layout", C.c_int32), ("n_real", C.c_int32), ("n_temps", C.c_int32),
                ("n_sets", C.c_int32), ("hot_start", C.c_int32), ("seed", C.c_uint64),
                ("stream", C.c_void_p)]


class spin_batch_item(C.Structure):
    _fields_ = [("lat", C.c_void_p), ("couplings", C.c_void_p), ("betas", C.c_void_p),
                ("E_series", C.c_void_p), ("M_series", C.c_void_p), ("Q_series", C.c_void_p),
                ("accepted", C.c_void_p), ("labels", C.c_void_p)]


class SpinError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """Loads libspin_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        p, i32, i64, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        L.spin_init.argtypes = [C.POINTER(p), C.POINTER(spin_desc), p, p]
        L.spin_sweep.argtypes = [p, p, p, i64, u64]
        L.spin_measure.argtypes = [p, p, p, p, p, p, p]
        L.spin_pt_swap.argtypes = [p, p, p, u64, p, p]
        L.spin_run.argtypes = [p, p, p, i64, i32, i32, p, p, p, p, p, p, p]
        L.spin_unpack_i8.argtypes = [p, p]
        L.spin_pack_i8.argtypes = [p, p]
        L.spin_rng_fill.argtypes = [u64, u32, u32, u32, u32, u32, u64, p, p]
        L.spin_rng_probe.argtypes = [u64, u32, u32, p, p]
        L.spin_pipe_probe.argtypes = [C.c_int, i32, u32, p, p, p, p]
        L.spin_describe.argtypes = [p, C.POINTER(spin_desc)]
        L.spin_sync.argtypes = [p]
        L.spin_heis_measure_noalloc.argtypes = [p, i32, i32, i32, p, p, p]
        L.spin_batch_run.argtypes = [p, C.c_int, i64, i32, i32, p]
        L.spin_batch_tune.argtypes = [p, C.c_int, i64, i32, i32, p, p]
        L.spin_set_batch_options.argtypes = [p, u64, i32, i32]
        L.spin_sweeps_done.argtypes = [p]
        L.spin_sweeps_done.restype = i64
        L.spin_pt_steps_done.argtypes = [p]
        L.spin_pt_steps_done.restype = i64
        L.spin_set_counters.argtypes = [p, i64, i64]
        L.spin_set_variant.argtypes = [p, i32]
        L.spin_set_update_order.argtypes = [p, i32, i32, i32]
        L.spin_set_msc_width.argtypes = [p, i32]
        L.spin_tune.argtypes = [p, p, p, i64, p, p]
        L.spin_slab_phase.argtypes = [p, i32, i32, i32, C.c_double, u64, u32, u32, i32, p]
        L.spin_slab_measure.argtypes = [p, i32, i32, p, p, p]
        L.spin_strerror.argtypes = [C.c_int]
        L.spin_strerror.restype = C.c_char_p
        L.spin_destroy.argtypes = [p]
        L.spin_destroy.restype = None
        for name in ("spin_init", "spin_sweep", "spin_measure", "spin_pt_swap", "spin_run",
                     "spin_unpack_i8", "spin_pack_i8", "spin_rng_fill", "spin_rng_probe", "spin_pipe_probe", "spin_sync",
                     "spin_set_counters", "spin_set_variant", "spin_batch_run", "spin_batch_tune",
                     "spin_set_batch_options", "spin_heis_measure_noalloc", "spin_set_update_order", "spin_set_msc_width", "spin_tune", "spin_slab_phase",
                     "spin_slab_measure", "spin_describe"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def spin_strerror(code):
    return lib().spin_strerror(code).decode()


def strerror(code):
    try:
        return spin_strerror(code)
    except RuntimeError:
        return str(code)


def _check(rc, what):
    if rc != SPIN_OK:
        raise SpinError(rc, what)
    return rc


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _host_doubles(values):
    arr = (C.c_double * len(values))(*[float(v) for v in values])
    return arr


# ------------------------------------------------------------------ argument checks
# The C ABI takes host beta arrays and device buffers without their lengths
# (they follow from the handle's descriptor), so the binding checks every
# array it passes against the descriptor before the call.
def spin_describe(h):
    d = spin_desc()
    _check(lib().spin_describe(h, C.byref(d)), "spin_describe")
    return d


def _shape(h):
    d = spin_describe(h)
    return d, d.L ** d.dim, d.n_sets * d.n_temps * d.n_real


def _bad(what, msg):
    raise SpinError(SPIN_EINVAL, f"{what}: {msg}")


def _need_betas(d, betas, what):
    if len(betas) != d.n_temps:
        _bad(what, f"{len(betas)} betas for {d.n_temps} temperature slots")


def _need(t, n, dtype, what, name):
    """t (if given) must be a contiguous CUDA tensor of dtype with >= n elements."""
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() < n:
        _bad(what, f"{name} must be a contiguous CUDA {dtype} tensor of at least {n} elements "
                   f"(got {t.dtype}, {t.numel()}, cuda={t.is_cuda})")


def _need_couplings(d, N, couplings, what):
    import torch
    if d.model != SPIN_EA:
        return
    if couplings is None:
        _bad(what, "EA handles need their couplings")
    if d.layout == SPIN_I8:
        _need(couplings, d.n_real * d.dim * N, torch.int8, what, "couplings")
    else:
        _need(couplings, (d.n_real // 32) * d.dim * N, torch.int32, what, "couplings")


def _n_meas(h, n_sweeps, measure_every):
    """Measurement rows a call writes: sweep counts reaching a multiple of
    measure_every between the handle's count now and after the call."""
    if measure_every <= 0:
        return 0
    cur = spin_sweeps_done(h)
    return (cur + n_sweeps) // measure_every - cur // measure_every


def _need_series(h, d, n_lat, rows, E, M, Q, Ef, Mf, accepted, what, labels=None):
    import torch
    _need(labels, n_lat, torch.int32, what, "labels")
    _need(E, rows * n_lat, torch.int64, what, "E")
    _need(M, rows * n_lat, torch.int64, what, "M")
    _need(Q, rows * d.n_temps * d.n_real, torch.int64, what, "Q")
    _need(Ef, rows * n_lat, torch.float64, what, "Ef")
    _need(Mf, 3 * rows * n_lat, torch.float64, what, "Mf")
    _need(accepted, d.n_sets * d.n_temps, torch.int64, what, "accepted")


# ------------------------------------------------------------------ ABI names
def spin_init(desc, spins, couplings=None):
    h = C.c_void_p()
    _check(lib().spin_init(C.byref(h), C.byref(desc), _ptr(spins), _ptr(couplings)), "spin_init")
    return h


def spin_sweep(h, couplings, betas, n_sweeps, seed):
    d, N, _ = _shape(h)
    _need_betas(d, betas, "spin_sweep")
    _need_couplings(d, N, couplings, "spin_sweep")
    return _check(lib().spin_sweep(h, _ptr(couplings), _host_doubles(betas), n_sweeps, seed),
                  "spin_sweep")


def spin_measure(h, couplings=None, E=None, M=None, Q=None, Ef=None, Mf=None):
    d, N, n_lat = _shape(h)
    _need_couplings(d, N, couplings, "spin_measure")
    _need_series(h, d, n_lat, 1, E, M, Q, Ef, Mf, None, "spin_measure")
    return _check(lib().spin_measure(h, _ptr(couplings), _ptr(E), _ptr(M), _ptr(Q), _ptr(Ef),
                                     _ptr(Mf)), "spin_measure")


def spin_pt_swap(h, couplings, betas, seed, accepted=None, labels=None):
    d, N, n_lat = _shape(h)
    _need_betas(d, betas, "spin_pt_swap")
    _need_couplings(d, N, couplings, "spin_pt_swap")
    _need_series(h, d, n_lat, 0, None, None, None, None, None, accepted, "spin_pt_swap", labels)
    return _check(lib().spin_pt_swap(h, _ptr(couplings), _host_doubles(betas), seed,
                                     _ptr(accepted), _ptr(labels)), "spin_pt_swap")


def spin_run(h, couplings, betas, n_sweeps, measure_every=0, pt_every=0, E=None, M=None,
             Q=None, Ef=None, Mf=None, accepted=None, labels=None):
    d, N, n_lat = _shape(h)
    _need_betas(d, betas, "spin_run")
    _need_couplings(d, N, couplings, "spin_run")
    rows = _n_meas(h, n_sweeps, measure_every) if n_sweeps > 0 else 0
    _need_series(h, d, n_lat, rows, E, M, Q, Ef, Mf, accepted, "spin_run", labels)
    return _check(lib().spin_run(h, _ptr(couplings), _host_doubles(betas), n_sweeps,
                                 measure_every, pt_every, _ptr(E), _ptr(M), _ptr(Q), _ptr(Ef),
                                 _ptr(Mf), _ptr(accepted), _ptr(labels)), "spin_run")


def spin_unpack_i8(h, out):
    import torch
    _, N, n_lat = _shape(h)
    _need(out, n_lat * N, torch.int8, "spin_unpack_i8", "out")
    return _check(lib().spin_unpack_i8(h, _ptr(out)), "spin_unpack_i8")


def spin_pack_i8(h, inp):
    import torch
    _, N, n_lat = _shape(h)
    _need(inp, n_lat * N, torch.int8, "spin_pack_i8", "in")
    return _check(lib().spin_pack_i8(h, _ptr(inp)), "spin_pack_i8")


def spin_rng_fill(seed, tag, colour, extra, lattice_id, sweep, count, out, stream=None):
    return _check(lib().spin_rng_fill(seed, tag, colour, extra, lattice_id, sweep, count,
                                      _ptr(out), stream), "spin_rng_fill")


def spin_rng_probe(seed, threads, calls, out, stream=None):
    return _check(lib().spin_rng_probe(seed, threads, calls, _ptr(out), stream), "spin_rng_probe")


def spin_pipe_probe(op, blocks_per_sm, iters, cycles, sink, stream=None):
    """Launches the instruction-throughput probe; returns the SM count."""
    sms = C.c_int32(0)
    _check(lib().spin_pipe_probe(op, blocks_per_sm, iters, _ptr(cycles), _ptr(sink), C.byref(sms), stream),
           "spin_pipe_probe")
    return sms.value


def _batch_items(items, n_sweeps=0, measure_every=0):
    """items: list of dicts with keys lat (handle), couplings, betas and the
    optional device tensors E, M, Q, accepted, labels (checked against each handle's
    descriptor).  Returns the ctypes array and the host beta arrays that must
    stay alive during the call."""
    arr = (spin_batch_item * len(items))()
    keep = []
    for k, it in enumerate(items):
        lat = it["lat"].value if hasattr(it["lat"], "value") else it["lat"]
        d, N, n_lat = _shape(lat)
        _need_betas(d, it["betas"], "spin_batch_run")
        _need_couplings(d, N, it.get("couplings"), "spin_batch_run")
        rows = _n_meas(lat, n_sweeps, measure_every) if n_sweeps > 0 else 0
        _need_series(lat, d, n_lat, rows, it.get("E"), it.get("M"), it.get("Q"), None, None,
                     it.get("accepted"), "spin_batch_run", it.get("labels"))
        b = _host_doubles(it["betas"])
        keep.append(b)
        dp = lambda key: it[key].data_ptr() if it.get(key) is not None else None
        arr[k] = spin_batch_item(lat, dp("couplings"), C.cast(b, C.c_void_p), dp("E"), dp("M"),
                                 dp("Q"), dp("accepted"), dp("labels"))
    return arr, keep


def spin_batch_run(items, n_sweeps, measure_every=0, pt_every=0, stream=None):
    arr, keep = _batch_items(items, n_sweeps, measure_every)
    return _check(lib().spin_batch_run(arr, len(items), n_sweeps, measure_every, pt_every, stream),
                  "spin_batch_run")


def spin_batch_tune(items, n_sweeps, measure_every=0, pt_every=0, stream=None):
    arr, keep = _batch_items(items)
    best = C.c_int32(0)
    _check(lib().spin_batch_tune(arr, len(items), n_sweeps, measure_every, pt_every, stream,
                                 C.byref(best)), "spin_batch_tune")
    return best.value


def spin_tune(h, couplings, betas, n_sweeps):
    """Runs the per-handle autotuner; returns (variant, tile) it chose."""
    d, N, _ = _shape(h)
    _need_betas(d, betas, "spin_tune")
    _need_couplings(d, N, couplings, "spin_tune")
    v, t = C.c_int32(0), C.c_int32(0)
    _check(lib().spin_tune(h, _ptr(couplings), _host_doubles(betas), n_sweeps, C.byref(v), C.byref(t)),
           "spin_tune")
    return v.value, t.value


def spin_set_batch_options(h, timeout_ns=0, ctas_per_sm=0, missing_arrivals=0):
    return _check(lib().spin_set_batch_options(h, timeout_ns, ctas_per_sm, missing_arrivals),
                  "spin_set_batch_options")


def spin_heis_measure_noalloc(spins, dim, L, n_lat, Ef=None, Mf=None, stream=None):
    """Heisenberg E and M into caller-owned tensors without any device
    allocation (the partial sums use a fixed array inside the library)."""
    import torch
    _need(spins, 4 * n_lat * L ** dim, torch.float32, "spin_heis_measure_noalloc", "spins")
    _need(Ef, n_lat, torch.float64, "spin_heis_measure_noalloc", "Ef")
    _need(Mf, 3 * n_lat, torch.float64, "spin_heis_measure_noalloc", "Mf")
    return _check(lib().spin_heis_measure_noalloc(_ptr(spins), dim, L, n_lat, _ptr(Ef), _ptr(Mf), stream),
                  "spin_heis_measure_noalloc")


def spin_sync(h):
    return _check(lib().spin_sync(h), "spin_sync")


def spin_sweeps_done(h):
    return int(lib().spin_sweeps_done(h))


def spin_pt_steps_done(h):
    return int(lib().spin_pt_steps_done(h))


def spin_set_counters(h, sweeps_done, pt_steps_done):
    return _check(lib().spin_set_counters(h, sweeps_done, pt_steps_done), "spin_set_counters")


def spin_set_variant(h, variant):
    return _check(lib().spin_set_variant(h, variant), "spin_set_variant")


def spin_set_update_order(h, order, tile=0, hits=1):
    return _check(lib().spin_set_update_order(h, order, tile, hits), "spin_set_update_order")


def spin_set_msc_width(h, width):
    return _check(lib().spin_set_msc_width(h, width), "spin_set_msc_width")


def spin_slab_phase(slab, L, y0, rows, beta, seed, lattice_id, sweep, colour, stream=None):
    return _check(lib().spin_slab_phase(_ptr(slab), L, y0, rows, float(beta), seed, lattice_id, sweep,
                                        colour, stream), "spin_slab_phase")


def spin_slab_measure(slab, L, rows, E, M, stream=None):
    return _check(lib().spin_slab_measure(_ptr(slab), L, rows, _ptr(E), _ptr(M), stream),
                  "spin_slab_measure")


def spin_destroy(h):
    lib().spin_destroy(h)
