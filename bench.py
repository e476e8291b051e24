#!/usr/bin/env python
"""Throughput of the checkerboard Metropolis sweep on GB300, in spin flips/ns.

Workload: 2D Ising ferromagnet, L = 16384 (2^28 spins per lattice), int8
spins, one lattice at each beta in {0.40, 0.4407, 0.50}, hot start, Philox
uniforms drawn in-kernel.  One step = SWEEPS_PER_STEP checkerboard sweeps of
all three lattices followed by the energy / magnetisation reduction.  The
1-bit coded layout of the same workload is timed too and reported beside
the main number.  A spin flip is one attempted Metropolis update.

Arms:
  (default)          the CUDA library through its C ABI on N GPUs (one
                     process per GPU; each rank runs its own three lattices,
                     weak scaling, no collective on the data path);
  --impl reference   the CPU oracle (tests' reference implementation) on the
                     host cores, on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L = 16384
BETAS = [0.40, 0.4407, 0.50]
SWEEPS_PER_STEP = 10
METRIC = "spin flips/ns, 2D Ising L=16384 checkerboard Metropolis (int8), 1 GB300"
UNIT = "flips/ns"
WORKLOAD = ("2D Ising ferromagnet L=16384 periodic, int8 spins, 3 lattices at beta "
            "0.40/0.4407/0.50, hot start, Philox4x32-10, %d sweeps + E/M reduction per step"
            % SWEEPS_PER_STEP)

# Algorithmic integer operations per attempted flip of the fused int8 sweep:
# Philox4x32-10 = 10 rounds x (2 wide 32x32 multiplies + 2 three-input XORs)
# per 4 uniforms = 10 per flip; the local field of 8 bytes at once (4 XOR+AND
# pairs, 3 adds, 2 shifted neighbour words, on 64-bit words) = 18 ops per 4
# active sites = 4.5 per flip; the decision (select threshold, compare, form
# the flip byte, merge) = 4 per flip; loads/stores of 2 bytes = 0.5.
OPS_PER_FLIP = 19.0
# Integer issue rate of one SM: 4 sub-partitions x 32 lanes per clock.
LANE_OPS_PER_CLK_PER_SM = 128

# DRAM traffic of one fused sweep launch (3 lattices share a launch) from the
# ncu capture summarised in profiles/, valid while the kernel source hash
# matches; otherwise the figure is reported as null.
FUSED_TRAFFIC_BYTES = None
FUSED_TRAFFIC_SRC_SHA = None


def kernel_sha():
    p = os.path.join(ROOT, "paper_1101_1427_gb300", "csrc", "fused2d.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


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
                 "--format=csv,noheader,nounits", "-lms", "200"],
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
def oracle_rate(seconds=10.0, Ls=1024, beta=0.4407):
    """The oracle as it stands (serial C, one core) on Ls x Ls lattices."""
    import oracle
    s = oracle.ising_init(2, Ls, 1, 0)
    oracle.ising_run(2, Ls, s, beta, 1, 0, 0, 1, series=False)  # load / warm
    flips, t0, k = 0, time.perf_counter(), 1
    while time.perf_counter() - t0 < seconds:
        oracle.ising_run(2, Ls, s, beta, 1, 0, k, 1, series=False)
        flips += Ls * Ls
        k += 1
    dt = time.perf_counter() - t0
    return flips / (dt * 1e9), flips, dt


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    Ls = 1024
    s = oracle.ising_init(2, Ls, 1, 0)
    for k in range(args.warmup):
        oracle.ising_run(2, Ls, s, BETAS[1], 1, 0, k, 1, series=False)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.ising_run(2, Ls, s, BETAS[1], 1, 0, args.warmup + k, 1, series=False)
    dt = time.perf_counter() - t0
    value = args.steps * Ls * Ls / (dt * 1e9)
    sample = "one sweep of a 1024^2 lattice at beta=0.4407 per step (same per-flip work)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
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

    lat = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_I8, n_temps=n_lat, seed=1 + rank)
    E = torch.empty(n_lat, dtype=torch.int64, device=dev)
    M = torch.empty(n_lat, dtype=torch.int64, device=dev)

    def step():
        B.spin_sweep(lat.h, None, BETAS, S, lat.seed)
        B.spin_measure(lat.h, None, E, M)

    for _ in range(args.warmup):
        step()
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = visible.split(",")[local_rank] if visible else local_rank
    clocks = ClockSampler(smi_index)
    clocks.start()
    barrier()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step()
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    if world > 1:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * args.steps * flips_per_step / (ms * 1e6)

    # dominant kernel alone: fused sweep launches (an even count, so no copy)
    n_k = 2 * S
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    k0.record(stream)
    B.spin_sweep(lat.h, None, BETAS, n_k, lat.seed)
    k1.record(stream)
    torch.cuda.synchronize()
    launch_ms = k0.elapsed_time(k1) / n_k
    flips_per_launch = n_lat * L * L

    # same workload in the 1-bit coded layout
    lat_msc = sp.Lattice(B.SPIN_ISING, 2, L, B.SPIN_MSC1, n_temps=n_lat, seed=1 + rank)
    B.spin_sweep(lat_msc.h, None, BETAS, S, lat_msc.seed)
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(max(1, args.steps // 2)):
        B.spin_sweep(lat_msc.h, None, BETAS, S, lat_msc.seed)
        B.spin_measure(lat_msc.h, None, E, M)
    m1.record(stream)
    torch.cuda.synchronize()
    msc_value = max(1, args.steps // 2) * flips_per_step / (m0.elapsed_time(m1) * 1e6)
    lat_msc.close()

    # end to end through the API with host buffers: every step copies the
    # lattices in from pinned memory and the lattices and observables out
    host_in = torch.empty(lat.spins.numel(), dtype=torch.int8).pin_memory()
    host_in.copy_(lat.spins.cpu())
    host_out = torch.empty_like(host_in).pin_memory()
    host_obs = torch.empty(2 * n_lat, dtype=torch.int64).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lat.spins.copy_(host_in, non_blocking=True)
        step()
        host_out.copy_(lat.spins, non_blocking=True)
        host_obs[:n_lat].copy_(E, non_blocking=True)
        host_obs[n_lat:].copy_(M, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e_value = world * args.steps * flips_per_step / (e2e_ms * 1e6)
    lat.close()

    if rank != 0:
        return
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 1800.0
    achieved = OPS_PER_FLIP * flips_per_launch / (launch_ms * 1e-3) / 1e9  # Gop/s
    peak = sms * LANE_OPS_PER_CLK_PER_SM * mhz * 1e6 / 1e9
    traffic = FUSED_TRAFFIC_BYTES if FUSED_TRAFFIC_SRC_SHA == kernel_sha() else None
    cpu_value, cpu_flips, cpu_s = oracle_rate(args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "betas": BETAS, "lattices_per_gpu": n_lat,
                   "sweeps_per_step": S, "layout": "int8, fused out-of-place sweep",
                   "l2": "inputs larger than L2 (3 x 256 MiB per GPU)",
                   "msc1_flips_per_ns": msc_value, "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "fused2d_kernel", "launch_ms": launch_ms,
                     "ops_per_flip": OPS_PER_FLIP,
                     "peak_basis": f"{sms} SMs x {LANE_OPS_PER_CLK_PER_SM} lane-ops/clk x "
                                   f"{mhz:.0f} MHz (sampled median)"},
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_flips} flips on 1024^2 lattices at beta=0.4407 "
                                   f"({cpu_s:.1f} s)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": host_in.numel(),
                "d2h_bytes_per_step": host_out.numel() + 8 * 2 * n_lat},
        "gpu_launches": args.steps * (S + 1),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
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
