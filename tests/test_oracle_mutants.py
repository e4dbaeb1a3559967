"""The oracle's pins catch plausible mistakes.

Each case below plants one plausible mistake in a copy of the oracle's C
source (a dropped term, a wrong sign or index, an off-by-one, a swapped
operand), builds it on the CPU, and runs the pin suites (test_oracle.py and
test_oracle_alt.py) against it in a fresh process.  Every mutant must make
them fail.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "vbdr_oracle.c")

MUTANTS = {
    "mix64_shift": ("z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;",
                    "z = (z ^ (z >> 28)) * 0x94d049bb133111ebULL;"),
    "H_low_bits": ("uint64_t hi32 = orc_mix64(x ^ orc_mix64(A)) >> 32;",
                   "uint64_t hi32 = orc_mix64(x ^ orc_mix64(A)) & 0xffffffffULL;"),
    "rho_off_by_one": ("if ((x >> bit) & 1u) return pos;",
                       "if ((x >> bit) & 1u) return pos + 1;"),
    "rho_no_cap": ("if (r > 32 - b) r = 32 - b;", ""),
    "vidx_right_bits": ("return x >> (32 - i);", "return x & ((1u << i) - 1u);"),
    "phyidx_seed_A1": ("uint64_t s1 = orc_H(i, 1ULL << 32, o->A0);",
                       "uint64_t s1 = orc_H(i, 1ULL << 32, o->A1);"),
    "active_le_k": ("static int IsActiveDR(const orc_t *o, uint8_t dr) { return dr < o->k; }",
                    "static int IsActiveDR(const orc_t *o, uint8_t dr) { return dr <= o->k; }"),
    "slide_no_saturation": ("if (*dr < o->dr_max) (*dr)++;", "(*dr)++;"),
    "gfast_lowest_set_bit": ("if ((o->bs[j] >> i) & 1u) lbp1 = i + 1; /* highest set bit */",
                             "if (((o->bs[j] >> i) & 1u) && lbp1 == 0) lbp1 = i + 1;"),
    "gfast_bs_not_cleared": ("      o->bs[j] = 0;\n", "\n"),
    "gsmall_age_before_read": (
        "      o->reg[j] = (uint8_t)GetLBP1BDR(o, j);\n      o->pcsa[j] = (uint8_t)PcsaBDR(o, j);\n"
        "      for (uint32_t r = 1; r <= o->R; ++r) SlideDR(o, &drv[r]);",
        "      for (uint32_t r = 1; r <= o->R; ++r) SlideDR(o, &drv[r]);\n"
        "      o->reg[j] = (uint8_t)GetLBP1BDR(o, j);\n      o->pcsa[j] = (uint8_t)PcsaBDR(o, j);"),
    "serial_no_reset": ("      o->now[j] = 0;\n", "\n"),
    "alpha_64": ("if (m == 64) return 0.709;", "if (m == 64) return 0.697;"),
    "lc_threshold": ("if (E <= 2.5 * m && V > 0)", "if (E <= 0.5 * m && V > 0)"),
    "noise_sign": ("double n = (Z * g / (Z - g)) * (n_g / g - n_Z / Z);",
                   "double n = (Z * g / (Z - g)) * (n_g / g + n_Z / Z);"),
    "noise_dropped": ("double n = (Z * g / (Z - g)) * (n_g / g - n_Z / Z);",
                      "double n = (Z * g / (Z - g)) * (n_g / g);"),
    "scale_swapped": ("double n = (Z * g / (Z - g)) * (n_g / g - n_Z / Z);",
                      "double n = (Z * g / (Z + g)) * (n_g / g - n_Z / Z);"),
    "harmonic_exponent": ("s += 1ULL << (32 - M);", "s += 1ULL << (31 - M);"),
    "dr_width_short": ("while ((1u << w) < k + 1) ++w;", "while ((1u << w) < k) ++w;"),
    # register-level state loading (batched workload)
    "load_min_fold": ("      if (v > o->reg[j]) o->reg[j] = v;", "      if (v < o->reg[j]) o->reg[j] = v;"),
    "load_no_zero_fill": ("  memset(o->reg, 0, (size_t)o->Z);\n  for (uint64_t h = 0; h < n; ++h) {",
                          "  for (uint64_t h = 0; h < n; ++h) {"),
    "load_ignores_offsets": ("      uint8_t v = vregs[offsets[h] + i];", "      uint8_t v = vregs[h * g + i];"),
    # LogLog / PCSA (pins in test_oracle_alt.py)
    "loglog_alpha_exponent": ("return pow(base, -m);", "return pow(base, m);"),
    "loglog_mean_not_divided": ("return orc_loglog_alpha(m) * m * exp2((double)L / m);",
                                "return orc_loglog_alpha(m) * m * exp2((double)L);"),
    "pcsa_phi_inverted": ("return m / 0.77351 * exp2((double)P / m);",
                          "return m * 0.77351 * exp2((double)P / m);"),
    "pcsa_highest_active": ("    if (!IsActiveDR(o, drv[r])) return r - 1;\n  return o->R;",
                            "    if (IsActiveDR(o, drv[r])) return r;\n  return 0;"),
    "pcsa_read_after_aging": (
        "      o->pcsa[j] = (uint8_t)PcsaBDR(o, j);\n      for (uint32_t r = 1; r <= o->R; ++r) SlideDR(o, &drv[r]);",
        "      for (uint32_t r = 1; r <= o->R; ++r) SlideDR(o, &drv[r]);\n      o->pcsa[j] = (uint8_t)PcsaBDR(o, j);"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(mut)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o",
                           str(so), str(c), "-lm"])
    return str(so)


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    so = _build(tmp_path, name, old, new)
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle.py"), os.path.join(HERE, "test_oracle_alt.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
