"""The oracle's pins reject plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), compiles it, and runs the pin tests against that
copy in a child process: the pins must fail.  Only mutations that keep every
memory access in bounds are planted.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pd_oracle.c")

MUTANTS = {
    "min_becomes_max": ("smin += (ca < cb) ? ca : cb;", "smin += (ca > cb) ? ca : cb;"),
    "window_count_off_by_one": ("? len - (uint32_t)k + 1u : 0u;", "? len - (uint32_t)k : 0u;"),
    "kmer_compared_on_k_minus_1_letters": (
        "memcmp(g_res_for_sort + a, g_res_for_sort + b, (size_t)g_k_for_sort)",
        "memcmp(g_res_for_sort + a, g_res_for_sort + b, (size_t)(g_k_for_sort - 1))"),
    "zero_overlap_is_candidate": ("if (s == 0) continue; /* not a candidate */", ""),
    "cross_multiplication_transposed": (
        "uint64_t l = (uint64_t)s1 * (uint64_t)d2, r = (uint64_t)s2 * (uint64_t)d1;",
        "uint64_t l = (uint64_t)s1 * (uint64_t)d1, r = (uint64_t)s2 * (uint64_t)d2;"),
    "ratio_compared_by_numerator": ("return (l > r) - (l < r);", "return (s1 > s2) - (s1 < s2);"),
    # Algorithm 3 tests the column maximum and membership in A_ji[k]; the two
    # are the same condition (J is symmetric), so only dropping both is a mistake.
    "reciprocal_checks_dropped": (
        "      if (cs == 0 || cmp_ratio(R->S[at], R->Den[at], cs, cd) != 0) continue; /* not the column max */\n"
        "      if (!contains(R->col_row, R->col_ptr[k], R->col_ptr[k + 1], (int32_t)l)) continue;\n",
        ""),
    "union_term_dropped": ("      smax += a->cnt[i];\n      ++i;\n    } else {", "      ++i;\n    } else {"),
    "alphabet_unchecked": ("if (!valid_letter(residues[i], alphabet)) {", "if (0) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant_c = tmp_path / "mutant.c"
    mutant_c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", str(so),
                           str(mutant_c)])
    env = dict(os.environ, PD_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
