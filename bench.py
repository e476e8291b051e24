#!/usr/bin/env python
"""Throughput of the checkerboard Metropolis sweep on GB300, in spin flips/ns.

Workload: 2D Ising ferromagnet, L = 16384 (2^28 spins per lattice), one
lattice at each beta in {0.40, 0.4407, 0.50}, hot start, one Philox uniform
per attempted flip drawn in-kernel.  One step = SWEEPS_PER_STEP checkerboard
sweeps of all three lattices followed by the energy / magnetisation
reduction.  The headline uses the 1-bit multi-spin-coded layout; the int8
layout of the same workload is timed too and reported beside it.  A spin
flip is one attempted Metropolis update.

Arms:
  (default)          the CUDA library through its C ABI on N GPUs (one
                     process per GPU; each rank runs its own three lattices,
                     weak scaling, no collective on the data path);
  --impl reference   the CPU oracle (the tests' reference implementation) on
                     the host cores, on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L = 16384
BETAS = [0.40, 0.4407, 0.50]
SWEEPS_PER_STEP = 50
METRIC = "spin flips/ns, 2D Ising L=16384 checkerboard Metropolis, 1 GB300"
UNIT = "flips/ns"
WORKLOAD = ("2D Ising ferromagnet L=16384 periodic, 3 lattices at beta 0.40/0.4407/0.50, "
            "hot start, Philox4x32-10 uniform per site, %d sweeps + E/M reduction per step "
            "(20 steps = the configuration's 1000 sweeps); 1-bit multi-spin-coded layout (int8 layout "
            "reported beside it)" % SWEEPS_PER_STEP)

# Roofline of the sweep: every attempted flip consumes one 32-bit Philox
# word, and Philox4x32-10 costs 20 wide (32x32->64) multiplies per 4 words,
# i.e. 5 per flip.  They run on the FMA-heavy pipe, which completes 32 wide
# multiplies per clock per SM (derived from the generator probe, which keeps
# that pipe 92% busy at 1.49 Philox calls per clock per SM).  The sweep's
# roof is therefore SMs x 32 x f_SM wide multiplies per second.
WIDE_MULS_PER_FLIP = 5
WIDE_MULS_PER_CLK_PER_SM = 32
# The other configurations' roofs, from algorithmic operation counts per
# attempted flip (counted from the algorithm, not from compiled code):
#  * Heisenberg update: one whole Philox call (20 wide multiplies); its
#    other classes -- about 60 FP32 operations (128 per clock per SM) and 5
#    MUFU / conversion operations (16 per clock) -- bind later.
#  * coded EA word-site (32 realisations, one shared uniform), on the ALU
#    pipe (64 three-input logic operations per clock per SM, measured 63.7):
#    sweep 28 = 5 Philox XORs (a quarter call) + 3 threshold compares + 6
#    bond terms s ^ s_j ^ J + 8 for the bit-sliced 6-input count + 5 for the
#    flip mask + 1 to apply it; measuring E and Q every sweep (the
#    tempering run of the configuration) adds 10 (3 bond terms and
#    carry-save counting for E, half of the overlap's XOR and count per set)
#    and the bitwise exchange about 1 (3 operations per word of an accepted
#    pair, half the pairs tried per sweep).  Its Philox multiplies (5 per 32
#    flips) bind far later.
HEIS_WIDE_MULS_PER_FLIP = 20
ALU_OPS_PER_CLK_PER_SM = 64
EA_SWEEP_ALU_PER_WORD = 28
EA_PT_ALU_PER_WORD = 28 + 10 + 1

# DRAM bytes of one phase launch of the coded sweep over the three lattices
# (one launch captured with ncu, summarised in profiles/), valid while the
# kernel's sources (comments removed) hash to KERNEL_TRAFFIC_SRC_SHA; otherwise reported as null.
KERNEL_TRAFFIC_BYTES = 100_702_464 + 10_737_664
KERNEL_TRAFFIC_SRC_SHA = "ca191803ce573804"


def kernel_sha():
    """Hash of the headline kernel's source code with its comments removed
    (comments cannot change the compiled kernel)."""
    h = hashlib.sha256()
    for f in ("msc2d.cu", "msc2d_block.cuh"):
        text = open(os.path.join(ROOT, "paper_1101_1427_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(text.encode())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l.split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
# The CPU baseline runs the oracle as it stands on the workload's own
# lattice: the L = 16384 lattice of slot 1 (beta = 0.4407) from the oracle's
# hot start (untimed), swept band by band (256 or 64 rows, colour 0 then
# colour 1 of the band) with the oracle's row-band sweep, which updates the
# rows in place with their global colours and Philox counters.
BAND_LID = 1  # lattice_id(0, 0, 1): slot 1 of the headline handle (seed 1)


def oracle_lattice():
    import oracle
    return oracle.ising_init(2, L, 1, oracle.lattice_id(0, 0, 1)).reshape(L, L)


def oracle_bands(s, rows, seconds=None, steps=None, first=0):
    """Band sweeps of s until `seconds` have passed or `steps` bands are
    done; returns (flips, seconds)."""
    import oracle
    bands = (L - 2) // rows
    flips, k, t0 = 0, first, time.perf_counter()
    while (steps is not None and k - first < steps) or (seconds is not None and time.perf_counter() - t0 < seconds):
        y0 = 1 + rows * (k % bands)
        for colour in (0, 1):
            oracle.slab_phase(L, y0, rows, s[y0 - 1:y0 + rows + 1], BETAS[1], 1,
                              oracle.lattice_id(0, 0, 1), k // bands, colour)
        flips += rows * L
        k += 1
    return flips, time.perf_counter() - t0


def oracle_rate(seconds=10.0):
    """The oracle (serial C, one core) on 256-row bands of the workload's lattice."""
    s = oracle_lattice()
    oracle_bands(s, 256, steps=1)  # load / warm
    flips, dt = oracle_bands(s, 256, seconds=seconds, first=1)
    return flips / (dt * 1e9), flips, dt


def oracle_omp_sweeps(s, first, count):
    """`count` full sweeps of the workload's lattice s on all host cores
    (the oracle's sweep with the rows of each colour phase shared among
    OpenMP threads); returns (flips, seconds, threads used)."""
    import oracle
    t0 = time.perf_counter()
    used = 0
    for k in range(count):
        _, used = oracle.omp_ising2d_sweeps(L, s, BETAS[1], 1, oracle.lattice_id(0, 0, 1), first + k, 1)
    return count * L * L, time.perf_counter() - t0, used


def oracle_omp_rate(seconds=10.0):
    s = oracle_lattice()
    oracle_omp_sweeps(s, 0, 1)  # warm
    flips, dt, k, used = 0, 0.0, 1, 0
    while dt < seconds:
        f, t, used = oracle_omp_sweeps(s, k, 1)
        flips, dt, k = flips + f, dt + t, k + 1
    return flips / (dt * 1e9), flips, dt, used


def run_reference(args, rank):
    if rank != 0:
        return
    s = oracle_lattice()
    oracle_omp_sweeps(s, 0, args.warmup)
    flips, dt, used = oracle_omp_sweeps(s, args.warmup, args.steps)
    value = flips / (dt * 1e9)
    sample = (f"per step one full checkerboard sweep of the workload's L=16384 lattice at beta=0.4407 "
              f"(slot 1, after the oracle's untimed hot start) on {used} host threads: the oracle's sweep "
              f"with the rows of each colour phase shared among OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_rooflines(side, i8_value, sms, mhz):
    """Roofline of every configuration's kernel from its algorithmic
    operations per attempted flip (see the constants at the top) and the
    pipe rates per clock per SM at the sampled SM clock."""
    f = mhz * 1e6
    philox2d = sms * WIDE_MULS_PER_CLK_PER_SM * f / WIDE_MULS_PER_FLIP / 1e9   # flips/ns
    heis = sms * WIDE_MULS_PER_CLK_PER_SM * f / HEIS_WIDE_MULS_PER_FLIP / 1e9
    ea_sweep = sms * ALU_OPS_PER_CLK_PER_SM * f * 32 / EA_SWEEP_ALU_PER_WORD / 1e9
    ea_pt = sms * ALU_OPS_PER_CLK_PER_SM * f * 32 / EA_PT_ALU_PER_WORD / 1e9
    mul_basis = f"{sms} SMs x {WIDE_MULS_PER_CLK_PER_SM} wide multiplies/clk x {mhz:.0f} MHz"
    alu_basis = f"{sms} SMs x {ALU_OPS_PER_CLK_PER_SM} logic ops/clk x {mhz:.0f} MHz"

    def line(value, peak, per_flip, basis, kernel):
        if value is None:
            return None
        return {"bound": "alu", "unit": "flips/ns", "achieved": value, "peak": peak, "frac": value / peak,
                "per_flip": per_flip, "peak_basis": basis, "kernel": kernel}

    out = {"2d_ising_L16384_i8": line(i8_value, philox2d, f"{WIDE_MULS_PER_FLIP} wide multiplies (Philox)",
                                      mul_basis, "msc2d_pack/phase/unpack (coded path of the int8 layout)")}
    for key, name in (("heisenberg_L128_fp32_flips_per_ns", "3d_heisenberg_L128_fp32"),
                      ("heisenberg_L128_fp32_fast_flips_per_ns", "3d_heisenberg_L128_fp32_fast")):
        out[name] = line(side.get(key), heis, f"{HEIS_WIDE_MULS_PER_FLIP} wide multiplies (one Philox call)",
                         mul_basis, "heis_resident_kernel (100-sweep calls)")
    out["3d_ea_L16_sweep"] = line(side.get("ea_L16_w32_sweep_flips_per_ns"), ea_sweep,
                                  f"{EA_SWEEP_ALU_PER_WORD}/32 logic ops", alu_basis, "msc_phase_kernel")
    out["3d_ea_L16_pt_per_handle"] = line(side.get("ea_L16_pt_plain_flips_per_ns"), ea_pt,
                                          f"{EA_PT_ALU_PER_WORD}/32 logic ops", alu_basis,
                                          "msc_phase_kernel + measure_msc_rows_kernel + pt kernels")
    out["3d_ea_L16_pt_batched"] = line(side.get("ea_L16_pt_batched_flips_per_ns"), ea_pt,
                                       f"{EA_PT_ALU_PER_WORD}/32 logic ops", alu_basis, "batch_kernel")
    # uneven batch: the roof of the mix is its total flips over the sum of
    # each unit's flips at its own roof
    n = 1
    ea_flips = sum(2 * T * R * Le ** 3 for Le, R, T in UNEVEN_EA) * n
    is_flips = sum(Li * Li for Li in UNEVEN_ISING) * n
    mix = (ea_flips + is_flips) / (ea_flips / ea_pt + is_flips / philox2d)
    for key, name in (("uneven_batch_batched_flips_per_ns", "uneven_batch_batched"),
                      ("uneven_batch_plain_flips_per_ns", "uneven_batch_per_handle")):
        out[name] = line(side.get(key), mix, "EA units as the tempering form, Ising units 5 wide multiplies",
                         f"{alu_basis}; {mul_basis}", "batch_kernel" if "batched" in name else "per-handle kernels")
    return {k: v for k, v in out.items() if v is not None}


# ---------------------------------------------------------------- GPU arm
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def side_configs(torch, sp, B, stream):
    """Short measurements of the other hot-path configurations (context for
    the headline): 3D Heisenberg L=128 and 2D L=4096 (FP32), and 3D EA L=16 with 1024
    realisations x 32 slots x 2 sets, exchange and overlap every sweep (and
    then E, M and Q), in the per-handle multi-launch form and in the batched
    persistent form;
    then the uneven batch in both forms, the 2D tempering benchmark, the
    double checkerboard and the 3D ferromagnet."""
    import numpy as np
    out = {}
    # Heisenberg lines are timed in equilibrium: right after the hot start
    # far more proposals are accepted (and written back) than later on
    lat = sp.Lattice(B.SPIN_HEISENBERG, 3, 128, B.SPIN_F32X4, seed=11)
    B.spin_sweep(lat.h, None, [0.693], 200, lat.seed)
    for variant, name in ((0, "heisenberg_L128_fp32"), (2, "heisenberg_L128_fp32_fast")):
        lat.set_variant(variant)
        B.spin_sweep(lat.h, None, [0.693], 4, lat.seed)
        a, b = _events(torch)
        a.record(stream)
        B.spin_sweep(lat.h, None, [0.693], 100, lat.seed)
        b.record(stream)
        torch.cuda.synchronize()
        out[name + "_flips_per_ns"] = 100 * 128 ** 3 / (a.elapsed_time(b) * 1e6)
    lat.close()
    # the paper's own Heisenberg study is 2D, L = 4096 (Sec. 4)
    lat = sp.Lattice(B.SPIN_HEISENBERG, 2, 4096, B.SPIN_F32X4, seed=13)
    B.spin_sweep(lat.h, None, [1.1], 50, lat.seed)
    for variant, name in ((0, "heisenberg2d_L4096_fp32"), (2, "heisenberg2d_L4096_fp32_fast")):
        lat.set_variant(variant)
        B.spin_sweep(lat.h, None, [1.1], 2, lat.seed)
        a, b = _events(torch)
        a.record(stream)
        B.spin_sweep(lat.h, None, [1.1], 20, lat.seed)
        b.record(stream)
        torch.cuda.synchronize()
        out[name + "_flips_per_ns"] = 20 * 4096 ** 2 / (a.elapsed_time(b) * 1e6)
    # ... in the paper's own GPU order: double checkerboard, 8 x 8 tiles, k = 100
    lat.set_update_order(B.SPIN_ORDER_DCB, 8, 100)
    for variant, name in ((0, "heisenberg2d_L4096_dcb_T8_k100_fp32"), (2, "heisenberg2d_L4096_dcb_T8_k100_fp32_fast")):
        lat.set_variant(variant)
        lat.set_counters(0, 0)
        B.spin_sweep(lat.h, None, [1.1], 100, lat.seed)
        a, b = _events(torch)
        a.record(stream)
        B.spin_sweep(lat.h, None, [1.1], 100, lat.seed)
        b.record(stream)
        torch.cuda.synchronize()
        out[name + "_flips_per_ns"] = 100 * 4096 ** 2 / (a.elapsed_time(b) * 1e6)
    lat.close()
    betas = list(1.0 / np.geomspace(0.9, 2.0, 32))
    ea = sp.Lattice(B.SPIN_EA, 3, 16, B.SPIN_MSC1, n_real=1024, n_temps=32, n_sets=2, seed=12)
    n = 40
    flips = n * 16 ** 3 * 1024 * 32 * 2
    ser = ea.series_buffers(n)
    acc = torch.zeros(64, dtype=torch.int64, device=stream.device)
    # the configuration's tempering run: exchange and overlap every sweep (the
    # exchange needs the energies, which are therefore recorded too); then
    # the same with the magnetisation measured as well
    for suffix, M in (("", None), ("_with_M", ser["M"])):
        B.spin_run(ea.h, ea.couplings, betas, 2, 1, 1, ser["E"], M, ser["Q"], None, None, acc)
        best = 1e30
        for _ in range(2):
            a, b = _events(torch)
            a.record(stream)
            B.spin_run(ea.h, ea.couplings, betas, n, 1, 1, ser["E"], M, ser["Q"], None, None, acc)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        out[f"ea_L16_pt{suffix}_plain_flips_per_ns"] = flips / (best * 1e6)
        item = [{"lat": ea.h, "couplings": ea.couplings, "betas": betas, "E": ser["E"], "M": M, "Q": ser["Q"],
                 "accepted": acc}]
        B.spin_batch_run(item, 2, 1, 1, stream.cuda_stream)
        best = 1e30
        for _ in range(2):
            a, b = _events(torch)
            a.record(stream)
            B.spin_batch_run(item, n, 1, 1, stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        ea.sync()
        out[f"ea_L16_pt{suffix}_batched_flips_per_ns"] = flips / (best * 1e6)
    # the same lattices with 64 realisations per shared uniform (Sec. 5, w = 64)
    ea.set_msc_width(64)
    for name, me in (("ea_L16_w64_sweep_flips_per_ns", 0), ("ea_L16_w64_pt_plain_flips_per_ns", 1)):
        B.spin_run(ea.h, ea.couplings, betas, 2, me, me, ser["E"] if me else None, ser["M"] if me else None,
                   ser["Q"] if me else None, None, None, acc if me else None)
        a, b = _events(torch)
        a.record(stream)
        B.spin_run(ea.h, ea.couplings, betas, n, me, me, ser["E"] if me else None, ser["M"] if me else None,
                   ser["Q"] if me else None, None, None, acc if me else None)
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = flips / (a.elapsed_time(b) * 1e6)
    ea.set_msc_width(32)
    a, b = _events(torch)
    a.record(stream)
    B.spin_run(ea.h, ea.couplings, betas, n, 0, 0, None, None, None, None, None, None)
    b.record(stream)
    torch.cuda.synchronize()
    out["ea_L16_w32_sweep_flips_per_ns"] = flips / (a.elapsed_time(b) * 1e6)
    ea.close()
    # the paper's own multi-spin-coding benchmark is the 2D glass, L = 16 (Sec. 5):
    # 16384 realisations x 32 temperatures x 2 sets (2^28 spins), sweeps only
    ea2 = sp.Lattice(B.SPIN_EA, 2, 16, B.SPIN_MSC1, n_real=16384, n_temps=32, n_sets=2, seed=14)
    flips2 = n * 16 ** 2 * 16384 * 32 * 2
    for width in (32, 64):
        ea2.set_msc_width(width)
        B.spin_run(ea2.h, ea2.couplings, betas, 2, 0, 0, None, None, None, None, None, None)
        a, b = _events(torch)
        a.record(stream)
        B.spin_run(ea2.h, ea2.couplings, betas, n, 0, 0, None, None, None, None, None, None)
        b.record(stream)
        torch.cuda.synchronize()
        out[f"ea2d_L16_w{width}_sweep_flips_per_ns"] = flips2 / (a.elapsed_time(b) * 1e6)
    ea2.close()
    out.update(uneven_batch(torch, sp, B, stream))
    out.update(ising_pt(torch, sp, B, stream))
    out.update(ising2d_small(torch, sp, B, stream))
    out.update(dcb(torch, sp, B, stream))
    out.update(ising3d(torch, sp, B, stream))
    return out


def ising3d(torch, sp, B, stream):
    """3D Ising ferromagnet (Sec. 3.6): one int8 lattice of L = 512 (2^27 sites,
    larger than L2) at the critical coupling, plain red-black sweeps and the
    double checkerboard with cubic tiles (T = 8, 16) and k = 100 hits."""
    out = {}
    L, n = 512, 10
    lat = sp.Lattice(B.SPIN_ISING, 3, L, B.SPIN_I8, seed=31)
    B.spin_sweep(lat.h, None, [0.2216544], 2, lat.seed)
    a, b = _events(torch)
    a.record(stream)
    B.spin_sweep(lat.h, None, [0.2216544], n, lat.seed)
    b.record(stream)
    torch.cuda.synchronize()
    out["ising3d_L512_i8_flips_per_ns"] = n * L ** 3 / (a.elapsed_time(b) * 1e6)
    # the paper's 3D GPU order: double checkerboard with 8^3 tiles, k = 100
    for T, k in ((8, 100), (16, 100)):
        lat.set_update_order(B.SPIN_ORDER_DCB, T, k)
        lat.set_counters(0, 0)
        B.spin_sweep(lat.h, None, [0.2216544], k, lat.seed)
        a, b = _events(torch)
        a.record(stream)
        B.spin_sweep(lat.h, None, [0.2216544], k, lat.seed)
        b.record(stream)
        torch.cuda.synchronize()
        out[f"ising3d_dcb_T{T}_k{k}_flips_per_ns"] = k * L ** 3 / (a.elapsed_time(b) * 1e6)
    lat.close()
    # small lattices: 20 int8 replicas of L = 16 near the critical coupling,
    # 200 sweeps in one call, resident kernel against the colour phases
    betas = [0.2216544] * 20
    for variant, name in ((3, "resident"), (0, "phases")):
        sm = sp.Lattice(B.SPIN_ISING, 3, 16, B.SPIN_I8, n_temps=20, seed=33)
        sm.set_variant(variant)
        B.spin_sweep(sm.h, None, betas, 10, sm.seed)
        a, b = _events(torch)
        a.record(stream)
        B.spin_sweep(sm.h, None, betas, 200, sm.seed)
        b.record(stream)
        torch.cuda.synchronize()
        out[f"ising3d_L16x20_{name}_flips_per_ns"] = 200 * 20 * 16 ** 3 / (a.elapsed_time(b) * 1e6)
        sm.close()
    return out


def dcb(torch, sp, B, stream):
    """The paper's own update order (Sec. 3.2): double checkerboard with
    multi-hit updates inside shared-memory tiles, on the three L=16384 int8
    lattices of the headline workload."""
    out = {}
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=len(BETAS), seed=21)
    for T, k in ((16, 100), (32, 100), (64, 10), (64, 100)):
        lat.set_update_order(B.SPIN_ORDER_DCB, T, k)
        lat.set_counters(0, 0)
        B.spin_sweep(lat.h, None, BETAS, k, lat.seed)
        a, b = _events(torch)
        a.record(stream)
        B.spin_sweep(lat.h, None, BETAS, k, lat.seed)
        b.record(stream)
        torch.cuda.synchronize()
        out[f"ising2d_dcb_T{T}_k{k}_flips_per_ns"] = k * len(BETAS) * L * L / (a.elapsed_time(b) * 1e6)
    lat.close()
    return out


def ising_pt_sizes(torch, sp, B, stream):
    """The tempering benchmark over lattice sizes (the paper plots its flip
    time against L, Sec. 6): 20 int8 replicas, beta in [0.1, 0.15], one
    exchange per 100 sweeps, with the resident kernel (L <= 128) and the
    fused pass (L >= 32)."""
    import numpy as np
    out = {}
    betas = list(np.linspace(0.1, 0.15, 20))
    for Lp in (16, 32, 64, 128, 256, 512, 1024, 2048):
        n = 400 if Lp <= 256 else 200
        for variant, name in ((3, "resident"), (1, "fused")):
            lat = sp.Lattice(B.SPIN_ISING, 2, Lp, B.SPIN_I8, n_temps=20, seed=70)
            try:
                lat.set_variant(variant)
            except B.SpinError:
                lat.close()
                continue
            B.spin_run(lat.h, None, betas, 100, 0, 100, None, None, None, None, None, None)
            a, b = _events(torch)
            a.record(stream)
            B.spin_run(lat.h, None, betas, n, 0, 100, None, None, None, None, None, None)
            b.record(stream)
            torch.cuda.synchronize()
            out[f"L{Lp}_{name}"] = round(n * 20 * Lp * Lp / (a.elapsed_time(b) * 1e6), 2)
            lat.close()
    return out


def ising2d_small(torch, sp, B, stream):
    """2D Ising L = 64, int8, beta = 0.4407, 1000 sweeps with E and M after
    every sweep (one spin_run call), with the resident kernel (which
    measures itself: one launch) and with the fused pass plus a separate
    measurement per sweep."""
    out = {}
    for variant, name in ((3, "resident"), (1, "fused")):
        lat = sp.Lattice(B.SPIN_ISING, 2, 64, B.SPIN_I8, seed=1)
        lat.set_variant(variant)
        ser = lat.series_buffers(1000)
        B.spin_run(lat.h, None, [0.4407], 20, 1, 0, ser["E"], ser["M"], None, None, None, None)
        a, b = _events(torch)
        a.record(stream)
        B.spin_run(lat.h, None, [0.4407], 1000, 1, 0, ser["E"], ser["M"], None, None, None, None)
        b.record(stream)
        torch.cuda.synchronize()
        out[f"ising2d_L64_1000sweeps_EM_every_sweep_{name}_flips_per_ns"] = 1000 * 64 * 64 / (a.elapsed_time(b) * 1e6)
        lat.close()
    return out


def ising_pt(torch, sp, B, stream):
    """The paper's tempering benchmark for the 2D ferromagnet (Sec. 6): 20
    int8 replicas at equally spaced beta in [0.1, 0.15], one exchange step
    per 100 (and per 10) sweeps; flips/ns counts spin flips of all replicas.
    Each size runs its default kernel: resident (whole lattice in one CTA)
    at L = 64, the fused pass at L = 2048."""
    import numpy as np
    out = {}
    betas = list(np.linspace(0.1, 0.15, 20))
    for Lp, every, n in ((64, 100, 400), (2048, 100, 200), (2048, 10, 200)):
        lat = sp.Lattice(B.SPIN_ISING, 2, Lp, B.SPIN_I8, n_temps=20, seed=70)
        B.spin_run(lat.h, None, betas, every, 0, every, None, None, None, None, None, None)
        a, b = _events(torch)
        a.record(stream)
        B.spin_run(lat.h, None, betas, n, 0, every, None, None, None, None, None, None)
        b.record(stream)
        torch.cuda.synchronize()
        lat.sync()
        out[f"ising2d_pt20_L{Lp}_every{every}_flips_per_ns"] = n * 20 * Lp * Lp / (a.elapsed_time(b) * 1e6)
        lat.close()
    return out


# Uneven batch: 3D EA lattices of five sizes (L, realisations, temperatures
# geometric in [0.8, 2.2], two replica sets) and five 2D Ising ferromagnets
# (1-bit coded layout).
UNEVEN_EA = [(8, 512, 24), (12, 256, 30), (16, 128, 36), (24, 64, 42), (32, 32, 48)]
UNEVEN_ISING = [256, 512, 1024, 2048, 4096]


def uneven_batch(torch, sp, B, stream, n=20):
    """The uneven batch with measurement and exchange every sweep, twice:
    plain per-handle calls (spin_run, several launches per sweep) and one
    graph-replayed batched launch after the autotuner has run; then checks
    that both sides reached identical lattices."""
    import numpy as np

    def build():
        side = []
        for k, (Le, R, T) in enumerate(UNEVEN_EA):
            lat = sp.Lattice(B.SPIN_EA, 3, Le, B.SPIN_MSC1, n_real=R, n_temps=T, n_sets=2, seed=50 + k)
            side.append((lat, list(1.0 / np.geomspace(0.8, 2.2, T))))
        for k, Li in enumerate(UNEVEN_ISING):
            side.append((sp.Lattice(B.SPIN_ISING, 2, Li, B.SPIN_MSC1, seed=60 + k), [0.4407]))
        return side

    flips = n * (sum(2 * T * R * Le ** 3 for Le, R, T in UNEVEN_EA) + sum(Li * Li for Li in UNEVEN_ISING))
    plain, batch = build(), build()
    sers = []
    for lat, betas in plain + batch:
        ser = lat.series_buffers(n)
        if lat.n_sets < 2:
            ser.pop("Q", None)
        acc = torch.zeros(lat.n_sets * lat.n_temps, dtype=torch.int64, device=stream.device)
        sers.append((ser, acc))

    def plain_run(k):
        for (lat, betas), (ser, acc) in zip(plain, sers):
            pt = 1 if lat.model == B.SPIN_EA else 0
            B.spin_run(lat.h, lat.couplings, betas, k, 1, pt, ser["E"], ser["M"], ser.get("Q"), None, None,
                       acc)

    items = [lat.batch_item(betas, ser, acc) for (lat, betas), (ser, acc) in zip(batch, sers[len(plain):])]
    plain_run(2)
    B.spin_batch_run(items, 2, 1, 1, stream.cuda_stream)
    best = B.spin_batch_tune(items, 4, 1, 1, stream.cuda_stream)
    graph = sp.BatchGraph(items, n, 1, 1)
    out = {}
    a, b = _events(torch)
    a.record(stream)
    plain_run(n)
    b.record(stream)
    torch.cuda.synchronize()
    out["uneven_batch_plain_flips_per_ns"] = flips / (a.elapsed_time(b) * 1e6)
    a.record(stream)
    graph.replay()
    b.record(stream)
    torch.cuda.synchronize()
    batch[0][0].sync()
    out["uneven_batch_batched_flips_per_ns"] = flips / (a.elapsed_time(b) * 1e6)
    out["uneven_batch_ctas_per_sm"] = best
    out["uneven_batch_identical"] = all(torch.equal(p.spins, q.spins) for (p, _), (q, _) in zip(plain, batch))
    for lat, _ in plain + batch:
        lat.close()
    return out


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1101_1427_gb300 as sp
    from paper_1101_1427_gb300 import _binding as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    S = SWEEPS_PER_STEP
    n_lat = len(BETAS)
    flips_per_step = S * n_lat * L * L

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(ms):
        if world > 1:
            tt = torch.tensor([ms], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt.item())
        return ms

    E = torch.empty(n_lat, dtype=torch.int64, device=dev)
    M = torch.empty(n_lat, dtype=torch.int64, device=dev)

    def make_step(lat):
        def step():
            B.spin_sweep(lat.h, None, BETAS, S, lat.seed)
            B.spin_measure(lat.h, None, E, M)
        return step

    def timed(step, k):
        barrier()
        a, b = _events(torch)
        a.record(stream)
        for _ in range(k):
            step()
        b.record(stream)
        barrier()
        return a.elapsed_time(b)

    # headline: 1-bit coded layout
    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=n_lat, seed=1 + rank)
    step = make_step(lat)
    for _ in range(args.warmup):
        step()
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = visible.split(",")[local_rank] if visible else local_rank
    clocks = ClockSampler(smi_index)
    clocks.start()
    ms = max_over_ranks(timed(step, args.steps))
    clk = clocks.stop()
    value = world * args.steps * flips_per_step / (ms * 1e6)

    # the dominant kernel alone: one colour phase over the three lattices per launch
    n_k = 2 * S
    torch.cuda.synchronize()
    a, b = _events(torch)
    a.record(stream)
    B.spin_sweep(lat.h, None, BETAS, S, lat.seed)
    b.record(stream)
    torch.cuda.synchronize()
    launch_ms = a.elapsed_time(b) / n_k
    flips_per_launch = n_lat * L * L // 2

    # end to end through the API with host buffers: every step copies the
    # coded lattices in from pinned memory and the lattices and observables
    # out, all inside the timed region.  Two handles (two device buffers)
    # take alternate steps; their sweeps run in order on one compute stream,
    # the host-to-device and device-to-host copies on two copy streams, tied
    # by events: the copy-in of a buffer waits for the copy-out of its
    # previous step, its sweeps wait for the copy-in, its copy-out waits for
    # the sweeps.  The copies of one step thus overlap the sweeps of the
    # other without the two handles' kernels competing for the SMs.
    host_in = torch.empty(lat.spins.numel(), dtype=lat.spins.dtype).pin_memory()
    host_in.copy_(lat.spins.cpu())
    spin_bytes = lat.spins.numel() * lat.spins.element_size()
    lat.close()
    comp, cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    pipes = []
    for k in range(2):
        h = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=n_lat, seed=1 + rank, stream=comp)
        Ek = torch.empty(n_lat, dtype=torch.int64, device=dev)
        Mk = torch.empty(n_lat, dtype=torch.int64, device=dev)
        pipes.append(dict(h=h, E=Ek, M=Mk, out=torch.empty_like(host_in).pin_memory(),
                          obs=torch.empty(2 * n_lat, dtype=torch.int64).pin_memory(),
                          copied_in=torch.cuda.Event(), swept=torch.cuda.Event(), copied_out=torch.cuda.Event()))
    torch.cuda.synchronize()
    for p in pipes:
        p["copied_out"].record(cout)
    e2e_count = [0]

    def e2e_step():
        p = pipes[e2e_count[0] % 2]
        e2e_count[0] += 1
        h = p["h"]
        cin.wait_event(p["copied_out"])  # the buffer's previous copy-out is done
        with torch.cuda.stream(cin):
            h.spins.copy_(host_in, non_blocking=True)
        p["copied_in"].record(cin)
        comp.wait_event(p["copied_in"])
        B.spin_sweep(h.h, None, BETAS, S, h.seed)
        B.spin_measure(h.h, None, p["E"], p["M"])
        p["swept"].record(comp)
        cout.wait_event(p["swept"])
        with torch.cuda.stream(cout):
            p["out"].copy_(h.spins, non_blocking=True)
            p["obs"][:n_lat].copy_(p["E"], non_blocking=True)
            p["obs"][n_lat:].copy_(p["M"], non_blocking=True)
        p["copied_out"].record(cout)

    def e2e_timed(k):
        barrier()
        a, b = _events(torch)
        a.record(stream)
        for st in (comp, cin, cout):
            st.wait_stream(stream)
        for _ in range(k):
            e2e_step()
        for st in (comp, cin, cout):
            stream.wait_stream(st)
        b.record(stream)
        barrier()
        return a.elapsed_time(b)

    for _ in range(2):
        e2e_step()
    e2e_ms = max_over_ranks(e2e_timed(args.steps))
    e2e_value = world * args.steps * flips_per_step / (e2e_ms * 1e6)
    for p in pipes:
        p["h"].close()

    # the int8 layout of the same workload (calls of 50 sweeps take the coded
    # path: pack, bit-sliced sweeps, unpack)
    lat8 = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=n_lat, seed=1 + rank)
    step8 = make_step(lat8)
    step8()
    k8 = max(3, args.steps // 3)
    i8_value = world * k8 * flips_per_step / (max_over_ranks(timed(step8, k8)) * 1e6)
    lat8.close()

    # the side configurations and the CPU baseline are single-GPU context: rank 0 at N = 1 only
    side = side_configs(torch, sp, B, stream) if rank == 0 and world == 1 and not args.no_side else {}
    if rank != 0:
        return
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    achieved = WIDE_MULS_PER_FLIP * flips_per_launch / (launch_ms * 1e-3) / 1e9  # Gmul/s
    peak = sms * WIDE_MULS_PER_CLK_PER_SM * mhz * 1e6 / 1e9
    traffic = KERNEL_TRAFFIC_BYTES if KERNEL_TRAFFIC_SRC_SHA == kernel_sha() else None
    cpu_baseline = None
    if world == 1:
        omp_value, omp_flips, omp_s, omp_threads = oracle_omp_rate(args.cpu_seconds)
        cpu_value, cpu_flips, cpu_s = oracle_rate(args.cpu_seconds)
        cpu_baseline = {"value": omp_value, "unit": UNIT, "cores": omp_threads, "kind": "oracle",
                        "sample": f"{omp_flips} flips: full checkerboard sweeps of the workload's L=16384 "
                                  f"lattice at beta=0.4407 ({omp_s:.1f} s, after the oracle's untimed hot start) "
                                  f"with the rows of each colour phase shared among {omp_threads} OpenMP threads "
                                  f"(os.cpu_count() = {os.cpu_count()})",
                        "single_core": {"value": cpu_value, "unit": UNIT, "cores": 1,
                                        "sample": f"{cpu_flips} flips in 256-row bands of the same lattice "
                                                  f"({cpu_s:.1f} s), the serial oracle"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 (1 bit per spin)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "betas": BETAS, "lattices_per_gpu": n_lat,
                   "sweeps_per_step": S, "layout": "1-bit synchronous multi-spin coding",
                   "i8_flips_per_ns": i8_value,
                   "l2": "coded lattices (96 MiB) fit in L2; int8 lattices (768 MiB) exceed it",
                   "e2e_form": "two handles take alternate steps, their sweeps in order on one compute stream, "
                               "copies on two copy streams ordered by events; each step copies its 3 lattices "
                               "in from pinned host memory and lattices + E, M out",
                   "parallelism": f"replicas x{world}", **side,
                   "rooflines": config_rooflines(side or {}, i8_value, sms, mhz)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gmul/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "msc2d_phase_kernel", "launch_ms": launch_ms,
                     "flips_per_launch": flips_per_launch,
                     "peak_basis": f"{sms} SMs x {WIDE_MULS_PER_CLK_PER_SM} wide multiplies/clk x "
                                   f"{mhz:.0f} MHz (sampled median); {WIDE_MULS_PER_FLIP} per flip"},
        "cpu_baseline": cpu_baseline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": spin_bytes,
                "d2h_bytes_per_step": spin_bytes + 8 * 2 * n_lat},
        "gpu_launches": args.steps * (2 * S + 1),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def pipe_rates(torch, B, stream, bpsm=8, iters=4096):
    """Operations per clock per SM of the instructions Philox and the updates
    are built from (spin_pipe_probe: 8 CTAs of 256 threads per SM, eight
    independent chains per thread): per SM, all its CTAs' operations over the
    span from the earliest start to the latest end of its CTAs in SM clocks;
    median over SMs."""
    import numpy as np
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clocks = torch.zeros(3 * sms * bpsm, dtype=torch.int64, device="cuda")
    sink = torch.zeros(sms * bpsm * 256, dtype=torch.int32, device="cuda")
    out = {}
    names = ("mul_wide", "mad_hi", "lop3", "iadd3", "ffma", "mufu_rsq")
    for op, nm in enumerate(names):
        B.spin_pipe_probe(op, bpsm, iters // 8, clocks, sink, stream.cuda_stream)  # warm-up
        B.spin_pipe_probe(op, bpsm, iters, clocks, sink, stream.cuda_stream)
        torch.cuda.synchronize()
        c = clocks.view(-1, 3).cpu().numpy()
        rates = []
        for m in np.unique(c[:, 2]):
            mine = c[c[:, 2] == m]
            rates.append(256 * 8 * iters * len(mine) / float(mine[:, 1].max() - mine[:, 0].min()))
        out[f"{nm}_per_clk_per_sm"] = round(float(np.median(rates)), 2)
    return out


def run_case(name):
    """One kernel family on a small case with few launches (for profilers):
    prints its throughput; not the benchmark line."""
    import numpy as np
    import torch

    import paper_1101_1427_gb300 as sp
    from paper_1101_1427_gb300 import _binding as B
    stream = torch.cuda.current_stream()
    a, b = _events(torch)
    if name in ("msc2d", "fused2d", "i8coded"):
        # fused2d: two-sweep calls of the int8 lattices (the fused pass);
        # i8coded: four-sweep calls (pack, coded sweeps, unpack)
        layout = B.SPIN_MSC1 if name == "msc2d" else B.SPIN_I8
        n = 4 if name == "i8coded" else 2
        lat = sp.Lattice(B.SPIN_ISING, 2, L, layout, n_temps=3, seed=1)
        B.spin_sweep(lat.h, None, BETAS, n, lat.seed)
        a.record(stream)
        B.spin_sweep(lat.h, None, BETAS, n, lat.seed)
        b.record(stream)
        flips = n * 3 * L * L
    elif name in ("ea", "ea_batch", "ea_measure"):
        betas = list(1.0 / np.geomspace(0.9, 2.0, 32))
        lat = sp.Lattice(B.SPIN_EA, 3, 16, B.SPIN_MSC1, n_real=1024, n_temps=32, n_sets=2, seed=1)
        if name == "ea_measure":
            # E, M and Q of every realisation, slot and set after two sweeps
            B.spin_sweep(lat.h, lat.couplings, betas, 2, lat.seed)
            lat.measure()
            a.record(stream)
            for _ in range(4):
                lat.measure()
            b.record(stream)
            flips = 4 * 2 ** 28  # spins read
        elif name == "ea":
            B.spin_sweep(lat.h, lat.couplings, betas, 2, lat.seed)
            a.record(stream)
            B.spin_sweep(lat.h, lat.couplings, betas, 2, lat.seed)
            b.record(stream)
            flips = 2 * 2 ** 28
        else:
            ser = lat.series_buffers(4)
            item = [lat.batch_item(betas, ser)]
            B.spin_batch_run(item, 2, 1, 1, stream.cuda_stream)
            a.record(stream)
            B.spin_batch_run(item, 4, 1, 1, stream.cuda_stream)
            b.record(stream)
            flips = 4 * 2 ** 28
    elif name == "ising3d":
        print(json.dumps({"case": name, **ising3d(torch, sp, B, stream)}), flush=True)
        return
    elif name == "dcb":
        print(json.dumps({"case": name, **dcb(torch, sp, B, stream)}), flush=True)
        return
    elif name == "ising_pt_sizes":
        print(json.dumps({"case": name, **ising_pt_sizes(torch, sp, B, stream)}), flush=True)
        return
    elif name == "ising_pt":
        print(json.dumps({"case": name, **ising_pt(torch, sp, B, stream), **ising2d_small(torch, sp, B, stream)}),
              flush=True)
        return
    elif name == "uneven":
        print(json.dumps({"case": name, **uneven_batch(torch, sp, B, stream, n=8)}), flush=True)
        return
    elif name in ("heis", "heis_fast"):
        # heis: the full-accuracy variant, heis_fast: the fast-math variant;
        # 20-sweep calls of L = 128, i.e. one launch of the resident kernel
        # each (the first, untimed, also takes the lattice off its hot start)
        lat = sp.Lattice(B.SPIN_HEISENBERG, 3, 128, B.SPIN_F32X4, seed=1)
        n = 20
        if name == "heis_fast":
            lat.set_variant(2)
        B.spin_sweep(lat.h, None, [0.693], n, lat.seed)
        a.record(stream)
        B.spin_sweep(lat.h, None, [0.693], n, lat.seed)
        b.record(stream)
        flips = n * 128 ** 3
    elif name == "pipes":
        print(json.dumps({"case": name, **pipe_rates(torch, B, stream)}), flush=True)
        return
    elif name == "heis_dcb":
        lat = sp.Lattice(B.SPIN_HEISENBERG, 2, 4096, B.SPIN_F32X4, seed=13)
        lat.set_update_order(B.SPIN_ORDER_DCB, 8, 100)
        B.spin_sweep(lat.h, None, [1.1], 100, lat.seed)
        a.record(stream)
        B.spin_sweep(lat.h, None, [1.1], 100, lat.seed)
        b.record(stream)
        flips = 100 * 4096 ** 2
    elif name == "rng":
        threads, calls = 152 * 2048, 256
        out = torch.empty(threads, dtype=torch.int32, device="cuda")
        B.spin_rng_probe(1, threads, calls, out, stream.cuda_stream)
        a.record(stream)
        B.spin_rng_probe(1, threads, calls, out, stream.cuda_stream)
        b.record(stream)
        flips = 4 * threads * calls  # words
    else:
        raise SystemExit(f"unknown case {name}")
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "per_ns": flips / (a.elapsed_time(b) * 1e6)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-side", action="store_true", help="skip the side configurations")
    ap.add_argument("--case", default=None,
                    help="run one kernel family briefly (msc2d, fused2d, i8coded, ea, ea_batch, ea_measure, ising_pt_sizes, heis, "
                         "heis_fast, heis_dcb, rng, pipes, uneven, ising_pt, dcb, ising3d)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.case:
        run_case(args.case)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
