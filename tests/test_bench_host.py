"""Host-side parts of the benchmark that need no GPU: the per-configuration
roofline arithmetic (peaks from the pipe rates per clock, fractions), the
validity of the recorded DRAM traffic of the headline kernel for the sources
as they stand, and the reference arm's JSON line (the oracle on the host
cores, one short step)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_config_rooflines_peaks_and_fractions():
    side = {"heisenberg_L128_fp32_flips_per_ns": 125.0, "heisenberg_L128_fp32_fast_flips_per_ns": 166.0,
            "ea_L16_w32_sweep_flips_per_ns": 9200.0, "ea_L16_pt_plain_flips_per_ns": 4000.0,
            "ea_L16_pt_batched_flips_per_ns": 4700.0, "uneven_batch_batched_flips_per_ns": 2500.0,
            "uneven_batch_plain_flips_per_ns": 1000.0}
    r = bench.config_rooflines(side, 1300.0, 152, 2070.0)
    f = 2070e6
    philox2d = 152 * 32 * f / 5 / 1e9  # 5 wide multiplies per flip at 32 per clock per SM
    heis = 152 * 32 * f / 20 / 1e9  # one Philox call (20 wide multiplies) per update
    ea_pt = 152 * 64 * f * 32 / 39 / 1e9  # 39 logic ops per 32-realisation word-site
    assert r["2d_ising_L16384_i8"]["peak"] == pytest.approx(philox2d)
    assert r["2d_ising_L16384_i8"]["frac"] == pytest.approx(1300.0 / philox2d)
    assert r["3d_heisenberg_L128_fp32_fast"]["peak"] == pytest.approx(heis)
    assert r["3d_heisenberg_L128_fp32_fast"]["frac"] == pytest.approx(166.0 / heis)
    assert r["3d_ea_L16_pt_batched"]["peak"] == pytest.approx(ea_pt)
    assert philox2d == pytest.approx(2014.0, rel=1e-3) and heis == pytest.approx(503.4, rel=1e-3)
    for line in r.values():
        if line is not None:
            assert 0.0 < line["frac"] < 1.0 and line["unit"] == "flips/ns"


def test_headline_traffic_record_matches_the_kernel_sources():
    """The DRAM traffic the bench line reports was measured on the headline
    kernel's current sources (comments aside); an edit of the kernel code
    makes the bench report null until the capture is repeated."""
    assert bench.kernel_sha() == bench.KERNEL_TRAFFIC_SRC_SHA


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "flips/ns" and line["higher_is_better"]
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "flips/ns", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
