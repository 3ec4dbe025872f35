"""Pins of the CPU oracle to things other than itself.

* hand-worked examples (tests/golden/, each citing the equations it follows);
* brute force on tiny random inputs: sum-min as a greedy matching of equal
  windows (multiset intersection), sum-max as an explicit union count, Best
  Hits as an exact maximum over Python Fractions, Bidirectional Best Hits as
  the set relation of Eq. (9);
* invariants of Eqs. (5), (8), (9): self-similarity, symmetry, bounds,
  sum-max identity, BBH symmetry and BBH subset of BH, invariance under a
  relabelling of the alphabet, equivariance under gene permutations, and a
  genome against its own copy;
* closed forms of the k rule reading (Eq. (4)).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import synth
from tests import _golden


# ---------------------------------------------------------------------------
# brute-force restatements (independent of the oracle's code)
# ---------------------------------------------------------------------------

def windows(g: bytes, k: int):
    return [g[p:p + k] for p in range(len(g) - k + 1)] if len(g) >= k else []


def brute_summin(a: bytes, b: bytes, k: int) -> int:
    """Size of a maximum matching between equal windows of a and b."""
    wb = windows(b, k)
    used = [False] * len(wb)
    s = 0
    for x in windows(a, k):
        for q, y in enumerate(wb):
            if not used[q] and x == y:
                used[q] = True
                s += 1
                break
    return s


def brute_summax(a: bytes, b: bytes, k: int) -> int:
    wa, wb = windows(a, k), windows(b, k)
    return sum(max(wa.count(w), wb.count(w)) for w in set(wa) | set(wb))


def brute_bh(q: bytes, targets, k: int):
    """Eq. (8) with exact rationals; candidates need a shared k-mer."""
    vals = {}
    for t, g in enumerate(targets):
        s = brute_summin(q, g, k)
        if s >= 1:
            vals[t] = Fraction(s, brute_summax(q, g, k))
    if not vals:
        return []
    best = max(vals.values())
    return sorted(t for t, v in vals.items() if v == best)


def brute_pair(rows, cols, k):
    row_bh = [brute_bh(a, cols, k) for a in rows]
    col_bh = [brute_bh(b, rows, k) for b in cols]
    bbh = sorted((a, b) for a in range(len(rows)) for b in row_bh[a] if a in col_bh[b])
    return row_bh, col_bh, bbh


def run_oracle(rows, cols, k, n_threads=1):
    ds = synth.from_strings([rows, cols])
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, k)
    return prof, oracle.pair(prof, ds.genome_ptr, 0, 1, n_threads)


def csr_lists(ptr, idx):
    return [sorted(idx[ptr[x]:ptr[x + 1]].tolist()) for x in range(len(ptr) - 1)]


# ---------------------------------------------------------------------------
# hand-worked examples
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fname", _golden.all_fixtures())
def test_golden(fname):
    g = _golden.load(fname)
    prof, R = run_oracle(g.rows, g.cols, g.k)
    nr = len(g.rows)
    assert [prof.La(a) for a in range(nr)] == g.La_rows
    assert [prof.La(nr + b) for b in range(len(g.cols))] == g.La_cols
    for gene, mv in g.mv.items():
        idx = (g.rows + g.cols).index(gene)
        kmers, cnt = prof.mv(idx)
        assert [(km.decode(), int(c)) for km, c in zip(kmers, cnt)] == mv
    S = [[(int(R.S[a, b]), int(R.Den[a, b])) for b in range(len(g.cols))] for a in range(nr)]
    assert S == g.S
    assert csr_lists(R.row_ptr, R.row_col) == g.row_bh
    assert csr_lists(R.col_ptr, R.col_row) == g.col_bh
    assert [tuple(x) for x in R.bbh.tolist()] == g.bbh


def test_golden_bbh_is_symmetric_in_genome_order():
    g = _golden.load("bh_k2_ties_empty.txt")
    _, R = run_oracle(g.rows, g.cols, g.k)
    _, Rt = run_oracle(g.cols, g.rows, g.k)
    assert sorted((b, a) for a, b in R.bbh.tolist()) == sorted(map(tuple, Rt.bbh.tolist()))


# ---------------------------------------------------------------------------
# brute force on tiny random inputs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_brute_force_tiny(seed, k):
    letters = [b"AC", b"ACD", b"ACDEFGHIKL", synth.ALPHABET][seed % 4]
    ds = synth.random_tiny(seed * 7 + k, n_genomes=3, max_genes=6, max_len=30, letters=letters)
    genes = [ds.gene(g) for g in range(ds.n_genes)]
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, k)
    for a in range(ds.n_genes):
        for b in range(ds.n_genes):
            s, d = prof.summin(a, b)
            assert s == brute_summin(genes[a], genes[b], k)
            assert d == brute_summax(genes[a], genes[b], k)
    gp = ds.genome_ptr
    for gi, gj in itertools.permutations(range(ds.n_genomes), 2):
        rows = genes[gp[gi]:gp[gi + 1]]
        cols = genes[gp[gj]:gp[gj + 1]]
        R = oracle.pair(prof, gp, gi, gj)
        row_bh, col_bh, bbh = brute_pair(rows, cols, k)
        assert csr_lists(R.row_ptr, R.row_col) == row_bh
        assert csr_lists(R.col_ptr, R.col_row) == col_bh
        assert [tuple(x) for x in R.bbh.tolist()] == bbh


def test_threads_do_not_change_results():
    ds = synth.generate(n_genomes=2, genes_per_genome=("fixed", 40), n_families=25,
                        length_dist=("uniform", 10, 80), core_frac=0.5, accessory_draw=None,
                        subst_max=0.2, indel_max=0.05, paralog_frac=0.1, singleton_frac=0.1,
                        seed=11)
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, 2)
    R1 = oracle.pair(prof, ds.genome_ptr, 0, 1, 1)
    R4 = oracle.pair(prof, ds.genome_ptr, 0, 1, 4)
    assert np.array_equal(R1.S, R4.S) and np.array_equal(R1.bbh, R4.bbh)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def _small_pangenome(seed=5, n=3, m=30):
    return synth.generate(n_genomes=n, genes_per_genome=("fixed", m), n_families=20,
                          length_dist=("uniform", 3, 70), core_frac=0.5, accessory_draw=None,
                          subst_max=0.3, indel_max=0.05, paralog_frac=0.1, singleton_frac=0.1,
                          seed=seed)


@pytest.mark.parametrize("k", [2, 3])
def test_invariants_summin(k):
    ds = _small_pangenome()
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, k)
    for a in range(ds.n_genes):
        La = prof.La(a)
        assert La == max(0, len(ds.gene(a)) - k + 1)
        s, d = prof.summin(a, a)
        assert (s, d) == (La, La)          # J(a, a) = 1 whenever La >= 1
        for b in range(0, ds.n_genes, 3):
            s, d = prof.summin(a, b)
            assert (s, d) == prof.summin(b, a)          # symmetry
            assert 0 <= s <= min(La, prof.La(b))        # bounds, hence 0 <= J <= 1
            assert d == La + prof.La(b) - s             # union identity


def test_invariants_bh_bbh():
    ds = _small_pangenome(seed=8)
    k = 2
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, k)
    gp = ds.genome_ptr
    for gi, gj in itertools.combinations(range(ds.n_genomes), 2):
        R = oracle.pair(prof, gp, gi, gj)
        Rt = oracle.pair(prof, gp, gj, gi)
        assert np.array_equal(R.S, Rt.S.T)
        # BBH relation symmetric under swapping the genomes
        assert sorted((b, a) for a, b in R.bbh.tolist()) == sorted(map(tuple, Rt.bbh.tolist()))
        # row Best Hits of (i, j) are the column Best Hits of (j, i)
        assert csr_lists(R.row_ptr, R.row_col) == csr_lists(Rt.col_ptr, Rt.col_row)
        rows = csr_lists(R.row_ptr, R.row_col)
        cols = csr_lists(R.col_ptr, R.col_row)
        for a, b in R.bbh.tolist():          # BBH within BH, both ways
            assert b in rows[a] and a in cols[b]
        for a in range(len(rows)):           # every hit is at the row maximum
            for b in rows[a]:
                assert R.S[a, b] >= 1
                assert int(R.S[a, b]) * int(R.row_best_den[a]) == int(R.row_best_s[a]) * int(R.Den[a, b])


def test_alphabet_relabelling_invariance():
    ds = _small_pangenome(seed=9)
    perm = np.random.default_rng(3).permutation(20)
    table = np.zeros(256, np.uint8)
    src = np.frombuffer(synth.ALPHABET, np.uint8)
    table[src] = src[perm]
    relabelled = synth.Pangenome(residues=table[ds.residues], gene_ptr=ds.gene_ptr,
                                 genome_ptr=ds.genome_ptr, family=ds.family)
    for k in (2, 3):
        P1 = oracle.Profiles(ds.residues, ds.gene_ptr, k)
        P2 = oracle.Profiles(relabelled.residues, relabelled.gene_ptr, k)
        R1 = oracle.pair(P1, ds.genome_ptr, 0, 2)
        R2 = oracle.pair(P2, ds.genome_ptr, 0, 2)
        assert np.array_equal(R1.S, R2.S) and np.array_equal(R1.Den, R2.Den)
        assert np.array_equal(R1.row_col, R2.row_col) and np.array_equal(R1.bbh, R2.bbh)


def test_gene_permutation_equivariance():
    ds = _small_pangenome(seed=10)
    k = 2
    genes = [ds.gene(g) for g in range(ds.n_genes)]
    gp = ds.genome_ptr
    rows, cols = genes[gp[0]:gp[1]], genes[gp[1]:gp[2]]
    rng = np.random.default_rng(4)
    pr, pc = rng.permutation(len(rows)), rng.permutation(len(cols))
    _, R = run_oracle(rows, cols, k)
    _, Rp = run_oracle([rows[x] for x in pr], [cols[x] for x in pc], k)
    assert np.array_equal(Rp.S, R.S[np.ix_(pr, pc)])
    inv_r, inv_c = np.argsort(pr), np.argsort(pc)
    mapped = sorted((int(inv_r[a]), int(inv_c[b])) for a, b in R.bbh.tolist())
    assert mapped == [tuple(x) for x in Rp.bbh.tolist()]


def test_genome_against_its_copy():
    ds = _small_pangenome(seed=12, n=1, m=40)
    k = 3
    genes = [ds.gene(g) for g in range(ds.n_genes)]
    _, R = run_oracle(genes, list(genes), k)
    # J(a, b) = 1 exactly when the multiplicity vectors coincide, so the BBH
    # relation pairs each gene that has a window with every gene of equal profile.
    prof_key = [tuple(sorted(windows(g, k))) for g in genes]
    expect = sorted((a, b) for a in range(len(genes)) for b in range(len(genes))
                    if prof_key[a] and prof_key[a] == prof_key[b])
    assert [tuple(x) for x in R.bbh.tolist()] == expect
    assert all((a, a) in set(expect) for a in range(len(genes)) if prof_key[a])


# ---------------------------------------------------------------------------
# k rule (reading of Eq. (4)) and input checks
# ---------------------------------------------------------------------------

def test_choose_k_closed_forms():
    for k in range(1, 15):
        assert oracle.choose_k(20 ** k) == k
        assert oracle.choose_k(20 ** k + 1) == k + 1
    assert oracle.choose_k(1) == 1
    assert oracle.choose_k(4 ** 10, alphabet=4) == 10


def test_rejects_letters_outside_alphabet():
    ds = synth.from_strings([[b"ACDB"], [b"ACD"]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.Profiles(ds.residues, ds.gene_ptr, 2)
    assert e.value.code == oracle.ERR_ALPHABET


@pytest.mark.parametrize("better_first", [True, False])
def test_bh_separates_ratios_closer_than_float_resolution(better_first):
    """Eq. (8) by exact comparison: targets at 60000/60001 and 59999/60000
    (equal as floats) give the larger alone; S and the denominators follow
    from letter counts at k = 1 (a multiset intersection)."""
    rng = np.random.default_rng(7)
    letters = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", np.uint8)
    a = rng.choice(letters, 60000)
    better = np.concatenate([a, letters[:1]])
    worse = a[:-1]
    genes = [a] + ([better, worse] if better_first else [worse, better])
    res = np.concatenate(genes).astype(np.uint8)
    gp = np.cumsum([0] + [len(g) for g in genes]).astype(np.int64)
    prof = oracle.Profiles(res, gp, 1)
    R = oracle.pair(prof, np.array([0, 1, 3], np.int32), 0, 1)
    counts = [np.bincount(g, minlength=256) for g in genes]
    s = [int(np.minimum(counts[0], counts[j]).sum()) for j in (1, 2)]
    assert R.S[0].tolist() == s
    ratios = [Fraction(s[j], len(genes[0]) + len(genes[j + 1]) - s[j]) for j in (0, 1)]
    assert sorted(ratios) == [Fraction(59999, 60000), Fraction(60000, 60001)]
    assert R.row_bh(0).tolist() == [int(np.argmax(ratios))] == [0 if better_first else 1]
