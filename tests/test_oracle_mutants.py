"""The oracle's pins reject plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), compiles it, and runs the pin tests against that
copy in a child process: the pins must fail.  Only mutations that keep every
memory access in bounds are planted.  The extensions (filters of Eqs. (6)-(7),
the nucleotide alphabet, paralogs, families) get their own mistakes, in the C
source or in the Python package, each checked against its own pin file.
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

# Mistakes in the extensions, each with the pin file that must reject it.
# C source (pd_oracle.c):
EXT_C_MUTANTS = {
    "directional_sums_swapped": ("      sa += x->cnt[i];\n      sb += y->cnt[j];\n",
                                 "      sa += y->cnt[j];\n      sb += x->cnt[i];\n", "test_oracle_filters.py"),
    "directional_sum_of_minima": ("      sa += x->cnt[i];\n",
                                  "      sa += x->cnt[i] < y->cnt[j] ? x->cnt[i] : y->cnt[j];\n",
                                  "test_oracle_filters.py"),
    "nucleotide_letter_wrong": ('static const char kNucleotide[] = "ACGT";', 'static const char kNucleotide[] = "ACGU";',
                                "test_oracle_nucleotide.py"),
}
# Python package (oracle/__init__.py):
PY_MUTANTS = {
    "theta_direction_flipped": ("if theta[0] and (la * theta[1] < theta[0] * lb or lb * theta[1] < theta[0] * la):",
                                "if theta[0] and (la * theta[1] > theta[0] * lb or lb * theta[1] > theta[0] * la):",
                                "test_oracle_filters.py"),
    "tau_against_gene_length": ("if pa * tau[1] < tau[0] * (la - k + 1) or pb * tau[1] < tau[0] * (lb - k + 1):",
                                "if pa * tau[1] < tau[0] * la or pb * tau[1] < tau[0] * lb:",
                                "test_oracle_filters.py"),
    "paralog_keeps_the_gene_itself": ("if b == a or s < 1:", "if s < 1:", "test_oracle_paralogs.py"),
    "family_label_of_the_parent": ("                        label[v] = s\n", "                        label[v] = u\n",
                                   "test_oracle_families.py"),
}


# Mistakes planted in oracle B (pd_oracle_b.c), each rejected by its pins
# against oracle A (test_oracle_b.py).
SRC_B = os.path.join(ROOT, "oracle", "pd_oracle_b.c")
B_MUTANTS = {
    "b_min_becomes_max": ("acc[b] += ca < cb ? ca : cb;", "acc[b] += ca > cb ? ca : cb;"),
    "b_window_count_off_by_one": ("const uint64_t La = len >= (uint64_t)k ? len - (uint64_t)k + 1 : 0;",
                                  "const uint64_t La = len > (uint64_t)k ? len - (uint64_t)k : 0;"),
    "b_own_genome_kept": ("if (gb == ga ? !J->own_genome : !J->target_genome[gb]) continue;",
                          "if (gb != ga && !J->target_genome[gb]) continue;"),
    "b_ties_dropped": ("if (ratio_cmp(s, den, best_s[gb], best_d[gb]) == 0) hit[n_hit++] = b;",
                       "if (ratio_cmp(s, den, best_s[gb], best_d[gb]) == 0 && (n_hit == 0 || "
                       "X->genome_of[hit[n_hit - 1]] != gb)) hit[n_hit++] = b;"),
    "b_denominator_without_overlap": ("const uint32_t s = acc[b], den = X->La[a] + X->La[b] - s;\n      if (best_s",
                                      "const uint32_t s = acc[b], den = X->La[a] + X->La[b];\n      if (best_s"),
    "b_bbh_one_sided": ("      if (!row_has(H, b, (int32_t)a)) continue;\n", ""),
    "b_multiplicity_ignored": ("X->mv_cnt[o] = (uint32_t)(q - p);", "X->mv_cnt[o] = 1u;"),
}


@pytest.mark.parametrize("name", sorted(B_MUTANTS))
def test_oracle_b_pins_reject_mutant(name, tmp_path):
    old, new = B_MUTANTS[name]
    src = open(SRC_B).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant_c = tmp_path / "mutant_b.c"
    mutant_c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant_b.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", str(so),
                           str(mutant_c)])
    env = dict(os.environ, PD_ORACLE_B_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", "not pan50x3000", os.path.join(ROOT, "tests", "test_oracle_b.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the oracle-B pins:\n{r.stdout[-2000:]}"


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


def _run_pins(pin_file, cwd, env):
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(cwd, "tests", pin_file)],
                          cwd=cwd, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", sorted(EXT_C_MUTANTS))
def test_extension_pins_reject_c_mutant(name, tmp_path):
    old, new, pin_file = EXT_C_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant_c = tmp_path / "mutant.c"
    mutant_c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", str(so),
                           str(mutant_c)])
    r = _run_pins(pin_file, ROOT, dict(os.environ, PD_ORACLE_LIB=str(so)))
    assert r.returncode != 0, f"mutant {name} survived {pin_file}:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_extension_pins_reject_python_mutant(name, tmp_path):
    """The oracle package is copied with one mistake into a scratch tree
    that links the tests and the input generator; the pins run there, on
    the unmodified compiled oracle."""
    import oracle
    old, new, pin_file = PY_MUTANTS[name]
    init = os.path.join(ROOT, "oracle", "__init__.py")
    src = open(init).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    lib = oracle.build()
    (tmp_path / "oracle").mkdir()
    (tmp_path / "oracle" / "__init__.py").write_text(src.replace(old, new))
    for d in ("tests", "paper_2510_23679_gb300"):
        os.symlink(os.path.join(ROOT, d), tmp_path / d)
    r = _run_pins(pin_file, str(tmp_path), dict(os.environ, PD_ORACLE_LIB=lib))
    assert r.returncode != 0, f"mutant {name} survived {pin_file}:\n{r.stdout[-2000:]}"


def test_scratch_tree_passes_unmutated(tmp_path):
    """The scratch tree itself is sound: the unmodified package passes."""
    import oracle
    lib = oracle.build()
    (tmp_path / "oracle").mkdir()
    (tmp_path / "oracle" / "__init__.py").write_text(open(os.path.join(ROOT, "oracle", "__init__.py")).read())
    for d in ("tests", "paper_2510_23679_gb300"):
        os.symlink(os.path.join(ROOT, d), tmp_path / d)
    r = _run_pins("test_oracle_families.py", str(tmp_path), dict(os.environ, PD_ORACLE_LIB=lib))
    assert r.returncode == 0, r.stdout[-2000:]
