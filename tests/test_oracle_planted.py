"""The oracle's pins catch plausible mistakes.

Each case below plants one plausible single mistake in a copy of
oracle/grng_oracle.cpp (a wrong constant, a swapped operand or index, a
dropped term, a transposed matrix entry, a wrong conversion), builds the copy,
and runs the oracle's CPU pins (tests/test_oracle_*.py, without the
known-answer fixtures, which the oracle wrote itself) against it: at least
one pin must fail.  The one mistake the CPU pins cannot see, the sign of the
MRG32k3a output combination, is pinned on the GPU against cuRAND
(tests/test_gpu_curand_pin.py) and is listed here without a CPU run.

The planted copies live in a temporary directory; the oracle itself is never
modified.
"""

import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "grng_oracle.cpp")
PINS = ["tests/test_oracle_philox.py", "tests/test_oracle_mrg.py",
        "tests/test_oracle_transforms.py", "tests/test_oracle_generate.py",
        "tests/test_oracle_icdf.py"]

# name -> (text in the oracle, planted replacement); each text occurs once
MUTANTS = {
    "philox_multiplier": ("const uint32_t PHILOX_M0 = 0xD2511F53u;",
                          "const uint32_t PHILOX_M0 = 0xD2511F55u;"),
    "philox_weyl_constant": ("const uint32_t PHILOX_W1 = 0xBB67AE85u;",
                             "const uint32_t PHILOX_W1 = 0xBB67AE87u;"),
    "philox_low_half_in_place_of_high": ("uint32_t n3 = lo0;", "uint32_t n3 = hi0;"),
    "philox_wrong_key_word": ("uint32_t n2 = hi0 ^ c[3] ^ k[1];",
                              "uint32_t n2 = hi0 ^ c[3] ^ k[0];"),
    "philox_nine_rounds": ("  for (int r = 0; r < 10; ++r) {\n    if (r > 0) {",
                           "  for (int r = 0; r < 9; ++r) {\n    if (r > 0) {"),
    "philox_key_bumped_before_first_round": ("    if (r > 0) {", "    if (r >= 0) {"),
    "philox_lane_order_reversed": ("return out[(unsigned)(g & 3)];",
                                   "return out[3u - (unsigned)(g & 3)];"),
    "philox_key_halves_swapped": (
        "uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};",
        "uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)seed};"),
    "mrg_multiplier_a12": ("const int64_t MRG_A12 = 1403580;", "const int64_t MRG_A12 = 1403581;"),
    "mrg_multiplier_a23": ("const int64_t MRG_A23 = 1370589;", "const int64_t MRG_A23 = 1370598;"),
    "mrg_modulus_m2": ("const int64_t MRG_M2 = 4294944443LL;",
                       "const int64_t MRG_M2 = 4294944437LL;"),
    "mrg_component2_wrong_lag": ("MRG_A21 * s.x2[2]", "MRG_A21 * s.x2[1]"),
    "mrg_seed_in_wrong_position": ("  s.x1[0] = 1;\n  s.x1[1] = 1;\n  s.x1[2] = (int64_t)(seed % (uint64_t)MRG_M1);",
                                   "  s.x1[2] = 1;\n  s.x1[1] = 1;\n  s.x1[0] = (int64_t)(seed % (uint64_t)MRG_M1);"),
    "mrg_companion_entry_transposed": ("  A.a[0][1] = 1;  // new x_{n-3} = old x_{n-2}",
                                       "  A.a[1][0] = 1;  // new x_{n-3} = old x_{n-2}"),
    "mrg_jump_multiplies_on_the_wrong_side": (
        "      if ((e[byte] >> bit) & 1) result = mat_mul(result, base, m);",
        "      if ((e[byte] >> bit) & 1) result = mat_mul(base, base, m);"),
    "u32_uniform_drops_a_bit": (
        "float u01_f32(uint32_t w) { return (float)std::ldexp((double)(w >> 8), -24); }",
        "float u01_f32(uint32_t w) { return (float)std::ldexp((double)(w >> 9), -23); }"),
    "u64_uniform_word_order": (
        "double u01_f64(uint32_t wa, uint32_t wb) {\n  uint64_t x = (((uint64_t)wa << 32) | (uint64_t)wb) >> 11;",
        "double u01_f64(uint32_t wa, uint32_t wb) {\n  uint64_t x = (((uint64_t)wb << 32) | (uint64_t)wa) >> 11;"),
    "range_without_clamp": ("  float r = a + t;\n  if (r >= b) r = std::nextafter(b, a);",
                            "  float r = a + t;"),
    "range_contracted_to_fma": ("  float t = d * u;\n  float r = a + t;",
                                "  float t = d * u;\n  float r = std::fmaf(d, u, a) + 0.0f * t;"),
    "box_muller_u1_closed_at_zero": (
        "float u01_f32_open0(uint32_t w) { return (float)std::ldexp((double)((w >> 8) + 1u), -24); }",
        "float u01_f32_open0(uint32_t w) { return (float)std::ldexp((double)(w >> 8), -24); }"),
    "box_muller_cos_sin_swapped": ("  *z0 = rho * std::cos(ang);\n  *z1 = rho * std::sin(ang);",
                                   "  *z0 = rho * std::sin(ang);\n  *z1 = rho * std::cos(ang);"),
    "box_muller_missing_factor_2": ("std::sqrt(-2.0L * std::log(u1))", "std::sqrt(-std::log(u1))"),
    "box_muller_angle_pi_not_2pi": ("long double ang = 2.0L * PI_L * u2;",
                                    "long double ang = PI_L * u2;"),
    "box_muller_pair_order": (
        "      u1 = (long double)u01_f32_open0(w[2 * k]);\n      u2 = (long double)u01_f32(w[2 * k + 1]);",
        "      u1 = (long double)u01_f32_open0(w[2 * k + 1]);\n      u2 = (long double)u01_f32(w[2 * k]);"),
    "gaussian_mean_sd_swapped": ("      long double v = mean + sd * z[j];",
                                 "      long double v = sd + mean * z[j];"),
    "icdf_midpoint_dropped": (
        "float u_mid_f32(uint32_t w) { return (float)std::ldexp(2.0 * (double)(w >> 9) + 1.0, -24); }",
        "float u_mid_f32(uint32_t w) { return (float)std::ldexp(2.0 * (double)(w >> 9) + 2.0, -24); }"),
    "icdf_upper_half_sign": ("return u <= 0.5L ? inv_phi_lower(u) : -inv_phi_lower(1.0L - u);",
                             "return u <= 0.5L ? inv_phi_lower(u) : inv_phi_lower(1.0L - u);"),
    "odd_count_does_not_round_to_pairs": ("  if (is_pair_dist(dist)) un = (un + 1u) / 2u * 2u;",
                                          "  if (is_pair_dist(dist)) un = un;"),
}

# Pinned on the GPU only (tests/test_gpu_curand_pin.py): both signs give
# statistically identical streams, so no CPU pin can tell them apart.
GPU_PINNED = {
    "mrg_output_sign": ("return (uint32_t)mod_floor(n1 - n2, MRG_M1);",
                        "return (uint32_t)mod_floor(n2 - n1, MRG_M1);"),
}


def test_each_planted_text_occurs_once():
    src = open(SRC).read()
    for name, (old, new) in {**MUTANTS, **GPU_PINNED}.items():
        assert src.count(old) == 1, name
        assert old != new, name


def _run_pins(name: str, old: str, new: str, base: str) -> int:
    d = os.path.join(base, name)
    os.makedirs(d, exist_ok=True)
    src = open(SRC).read().replace(old, new)
    path = os.path.join(d, "grng_oracle.cpp")
    with open(path, "w") as f:
        f.write(src)
    env = dict(os.environ, GRNG_ORACLE_SRC=path)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", *PINS], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return r.returncode


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(_run_pins, name, old, new, str(tmp_path))
                for name, (old, new) in MUTANTS.items()}
        codes = {name: f.result() for name, f in futs.items()}
    survivors = [name for name, rc in codes.items() if rc == 0]
    assert not survivors, f"planted mistakes no CPU pin caught: {survivors}"
    # a failing pin, not a build or collection error (exit code 1 = tests failed)
    assert all(rc == 1 for rc in codes.values()), codes


def test_unplanted_copy_passes_the_pins(tmp_path):
    """The harness itself: an unmodified copy passes every pin."""
    assert _run_pins("unmodified", "", "", str(tmp_path)) == 0
