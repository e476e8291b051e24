"""The pins must catch plausible mistakes in the oracle: each case plants
one mistake in a copy of the oracle's C source (on the CPU, in a temporary
directory), builds it, and checks that the named pin tests fail with it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spin_oracle.c")

MUTANTS = {
    "metropolis_sign": ("int dE = 2 * s[i] * h;", "int dE = -2 * s[i] * h;",
                        "tests/test_oracle_ising.py::test_mc_4x4_matches_enumeration"),
    "threshold_index": ("(uint32_t)(i >> 1));\n        flip = r < thr[dE / 4];",
                        "(uint32_t)(i >> 1));\n        flip = r < thr[dE / 4 - (dE > 4)];",
                        "tests/test_oracle_ising.py::test_mc_4x4_matches_enumeration"),
    "backward_coupling": ("int j_dn = J ? J[d * n + dn] : 1;", "int j_dn = J ? J[d * n + i] : 1;",
                          "tests/test_oracle_ising.py::test_mc_ea_matches_enumeration"),
    "colour_order": ("for (int colour = 0; colour < 2; ++colour) {\n    for (int64_t i = 0; i < n; ++i) {\n      if (or_colour(dim, L, i) != colour) continue;\n      int h = or_local_field",
                     "for (int colour = 1; colour >= 0; --colour) {\n    for (int64_t i = 0; i < n; ++i) {\n      if (or_colour(dim, L, i) != colour) continue;\n      int h = or_local_field",
                     "tests/test_oracle_ising.py::test_one_sweep_flip_frequencies_match_exact_probabilities"),
    "pt_sign": ("if (dbeta * (double)dE >= 0.0) {", "if (dbeta * (double)dE <= 0.0) {",
                "tests/test_oracle_pt_heis.py::test_pt_slot_marginals_and_swap_rates_match_exact"),
    "heis_energy_sign": ("dE -= (nv[k] - s[3 * i + k]) * h[k];", "dE += (nv[k] - s[3 * i + k]) * h[k];",
                         "tests/test_oracle_pt_heis.py::test_heis_chain_correlation_matches_langevin"),
    "heis_proposal": ("double z = 2.0 * u1 - 1.0;", "double z = u1;",
                      "tests/test_oracle_pt_heis.py::test_heis_infinite_temperature_gives_uniform_proposals"),
    "philox_word": ("uint32_t n2 = hi0 ^ c3 ^ k1;", "uint32_t n2 = hi0 ^ c1 ^ k1;",
                    "tests/test_oracle_rng.py::test_philox_matches_curand_host_generator"),
    "dcb_symmetric_order": ("const int first = (symmetric && (M & 1u)) ? 1 : 0;",
                            "const int first = (symmetric && !(M & 1u)) ? 1 : 0;",
                            "tests/test_oracle_dcb.py::test_one_compound_matches_exact_distribution"),
    "dcb_fine_colour_order": ("for (int colour = 0; colour < 2; ++colour) {\n          for (int64_t i = 0; i < n; ++i) {\n            const int x",
                              "for (int colour = 1; colour >= 0; --colour) {\n          for (int64_t i = 0; i < n; ++i) {\n            const int x",
                              "tests/test_oracle_dcb.py::test_one_compound_matches_exact_distribution"),
    "dcb_tile_colour": ("if (((x / T + y / T + z / T) & 1) != coarse) continue;",
                        "if (((x % T + y / T + z / T) & 1) != coarse) continue;",
                        "tests/test_oracle_dcb.py::test_one_compound_matches_exact_distribution"),
    "dcb3_tile_colour_without_z": ("if (((x / T + y / T + z / T) & 1) != coarse) continue;",
                                   "if (((x / T + y / T) & 1) != coarse) continue;",
                                   "tests/test_oracle_dcb.py::test_3d_zero_temperature_order_matches_numpy"),
    "dcb3_missing_threshold": ("const int64_t n = or_nsites(dim, L);\n  uint32_t thr[4] = {0, 0, 0, 0};\n  for (int m = 1; m <= dim; ++m)",
                               "const int64_t n = or_nsites(dim, L);\n  uint32_t thr[4] = {0, 0, 0, 0};\n  for (int m = 1; m < dim; ++m)",
                               "tests/test_oracle_dcb.py::test_3d_one_compound_matches_exact_distribution"),
    "overlap_one_replica_twice": ("q += s0[i] * s1[i];", "q += s0[i] * s0[i];",
                                  "tests/test_oracle_pt_heis.py::test_overlap_second_moment_matches_enumeration"),
    "overlap_sum_not_product": ("q += s0[i] * s1[i];", "q += s0[i] + s1[i];",
                                "tests/test_oracle_pt_heis.py::test_overlap_second_moment_matches_enumeration"),
    "magnetisation_sign": ("for (int64_t i = 0; i < n; ++i) m += s[i];",
                           "for (int64_t i = 0; i < n; ++i) m -= s[i];",
                           "tests/test_oracle_ising.py::test_mc_magnetisation_and_energy_match_yang_and_onsager"),
    "dcb_hit_words": ("const uint32_t sweep = M * (uint32_t)k + (uint32_t)h;",
                      "const uint32_t sweep = M * (uint32_t)k;",
                      "tests/test_oracle_dcb.py::test_one_compound_matches_exact_distribution"),
    "pt_labels_half_exchanged": ("labels[t + 1] = tl;", "labels[t + 1] = labels[t];",
                                 "tests/test_oracle_pt_heis.py::test_pt_labels_follow_the_configurations"),
    "heis_magnetisation_drops_z": ("for (int k = 0; k < 3; ++k) m[k] += s[3 * i + k];",
                                   "for (int k = 0; k < 2; ++k) m[k] += s[3 * i + k];",
                                   "tests/test_oracle_pt_heis.py::test_heis_magnetisation_second_moment"),
}


# where a line occurs in several functions, the mistake is planted in the
# function named here (its first occurrence after the function's signature)
SCOPES = {
    "dcb_symmetric_order": "void or_dcb_sweeps_dim(",
    "dcb_fine_colour_order": "void or_dcb_sweeps_dim(",
    "dcb_tile_colour": "void or_dcb_sweeps_dim(",
    "dcb3_tile_colour_without_z": "void or_dcb_sweeps_dim(",
    "dcb_hit_words": "void or_dcb_sweeps_dim(",
    "heis_dcb_hit_words": "void or_heis_dcb_sweeps(",
    "heis_dcb_renorm_rule": "void or_heis_dcb_sweeps(",
}
MUTANTS.update({
    "heis_dcb_hit_words": ("const uint32_t sweep = M * (uint32_t)k + (uint32_t)h;",
                           "const uint32_t sweep = M * (uint32_t)k;",
                           "tests/test_oracle_dcb.py::test_heis_dcb_infinite_temperature_keeps_the_last_proposal"),
    "heis_dcb_renorm_rule": ("after / (uint64_t)renorm_every > before / (uint64_t)renorm_every",
                             "after % (uint64_t)renorm_every == 0",
                             "tests/test_oracle_dcb.py::test_heis_dcb_renormalises_when_a_move_passes_a_multiple"),
})


def _plant(src, name, old, new):
    scope = SCOPES.get(name)
    if scope is None:
        assert src.count(old) == 1, name
        return src.replace(old, new)
    start = src.index(scope)
    pos = src.index(old, start)
    return src[:pos] + new + src[pos + len(old):]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new, target = MUTANTS[name]
    src = open(SRC).read()
    mut = tmp_path / "mutant.c"
    mut.write_text(_plant(src, name, old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    str(mut), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, SPIN_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        target], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if "skipped" in r.stdout and "failed" not in r.stdout:
        pytest.skip("pin skipped on this host")
    assert r.returncode != 0, f"mutant {name} survived:\n{r.stdout[-2000:]}"
