"""Pins of oracle B (pd_oracle_b.c: inverted index walked by host threads)
against oracle A (pd_oracle.c: the dense S_ij of each genome pair, itself
pinned to the paper's definitions in test_oracle_pins.py).  The two share no
code; equality is bit-exact: every Best Hit set with its sum-min values in
both directions of every compared genome pair, and every BBH pair."""
import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import synth


def _rows_towards(rp, cols, s, rows, t0, t1):
    out = []
    for a in rows:
        c = cols[rp[a]:rp[a + 1]]
        sel = (c >= t0) & (c < t1)
        out.append(((c[sel] - t0).tolist(), s[rp[a]:rp[a + 1]][sel].tolist()))
    return out


def _check_pair_against_a(ds, k, gi, gj, rp, cols, s, bbh, alphabet=20):
    """Oracle B's whole-dataset result restricted to (gi, gj) equals oracle A on that pair."""
    gp = ds.genome_ptr
    R = oracle.pair_for_dataset(ds, gi, gj, k, n_threads=oracle.default_threads(), alphabet=alphabet)
    i0, i1, j0, j1 = int(gp[gi]), int(gp[gi + 1]), int(gp[gj]), int(gp[gj + 1])
    fwd = _rows_towards(rp, cols, s, range(i0, i1), j0, j1)
    assert [c for c, _ in fwd] == [R.row_bh(a).tolist() for a in range(i1 - i0)], (gi, gj)
    assert [v for _, v in fwd] == [[int(R.S[a, b]) for b in R.row_bh(a)] for a in range(i1 - i0)], (gi, gj)
    rev = _rows_towards(rp, cols, s, range(j0, j1), i0, i1)
    assert [c for c, _ in rev] == [R.col_bh(b).tolist() for b in range(j1 - j0)], (gi, gj)
    lo, hi = (gi, gj) if gi < gj else (gj, gi)
    sel = (bbh[:, 0] >= gp[lo]) & (bbh[:, 0] < gp[lo + 1]) & (bbh[:, 1] >= gp[hi]) & (bbh[:, 1] < gp[hi + 1])
    got = (bbh[sel] - [int(gp[lo]), int(gp[hi])]).tolist()
    want = R.bbh.tolist() if gi < gj else sorted([b, a] for a, b in R.bbh.tolist())
    assert got == want, (gi, gj)


def test_every_pair_of_pan4x250_equals_oracle_a():
    ds = synth.workload("pan4x250")
    k = oracle.choose_k(ds.n_residues)
    idx = oracle.IndexB(ds, k)
    rp, cols, s, bbh = oracle.all_pairs_b(idx)
    for gi in range(ds.n_genomes):
        for gj in range(ds.n_genomes):
            if gi != gj:
                _check_pair_against_a(ds, k, gi, gj, rp, cols, s, bbh)
    assert np.array_equal(bbh.astype(np.int64), oracle.all_pairs_bbh(ds, k, oracle.default_threads()))


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_datasets_equal_oracle_a(seed):
    ds = synth.random_tiny(seed, n_genomes=3 + seed % 2, max_genes=7, max_len=30,
                           letters=b"ACDEFG" if seed % 2 else b"ACD")
    for k in (1, 2, 3):
        idx = oracle.IndexB(ds, k)
        rp, cols, s, bbh = oracle.all_pairs_b(idx)
        for gi in range(ds.n_genomes):
            for gj in range(ds.n_genomes):
                if gi != gj:
                    _check_pair_against_a(ds, k, gi, gj, rp, cols, s, bbh)


def test_sampled_pan50x3000_pairs_equal_oracle_a():
    """Two genome pairs of the 50-genome workload, profiled as two-genome
    datasets (Best Hits between two genomes do not depend on the others)."""
    ds = synth.workload("pan50x3000")
    k = oracle.choose_k(ds.n_residues)
    assert k == 6
    for gi, gj in ((7, 31), (48, 2)):
        sub = ds.subset([gi, gj])
        rp, cols, s, bbh = oracle.all_pairs_b(oracle.IndexB(sub, k))
        _check_pair_against_a(sub, k, 0, 1, rp, cols, s, bbh)


def test_target_lists_and_own_genome():
    """Listed queries towards listed genomes give the matching slices of the
    all-pairs rows; the own-genome mode gives the within-genome Best Hits of
    oracle A (the gene itself excluded)."""
    ds = synth.workload("pan4x250")
    k = oracle.choose_k(ds.n_residues)
    idx = oracle.IndexB(ds, k)
    rp, cols, s, _ = oracle.all_pairs_b(idx)
    gp = ds.genome_ptr
    q = np.arange(int(gp[1]), int(gp[2]), dtype=np.uint32)  # genes of genome 1
    for targets in ([3], [0, 2]):
        trp, tcols, ts = oracle.best_hits_b(idx, q, targets=targets)
        for x, a in enumerate(q):
            row, sv = cols[rp[a]:rp[a + 1]], s[rp[a]:rp[a + 1]]
            sel = np.isin(np.searchsorted(gp, row, side="right") - 1, targets)
            assert tcols[trp[x]:trp[x + 1]].tolist() == row[sel].tolist()
            assert ts[trp[x]:trp[x + 1]].tolist() == sv[sel].tolist()
    want = oracle.paralog_hits(ds, k, oracle.default_threads())
    prp, pcols, ps = oracle.best_hits_b(idx, np.arange(ds.n_genes, dtype=np.uint32), targets=[], own_genome=True)
    got = [(pcols[prp[a]:prp[a + 1]].tolist(), ps[prp[a]:prp[a + 1]].tolist()) for a in range(ds.n_genes)]
    assert got == [(c, v) for c, v in want]


def test_nucleotide_alphabet_equals_oracle_a():
    ds = synth.workload("nt8x600").subset([0, 3, 5])
    k = oracle.choose_k(ds.n_residues, alphabet=4)
    rp, cols, s, bbh = oracle.all_pairs_b(oracle.IndexB(ds, k, alphabet=4))
    for gi, gj in ((0, 1), (2, 0)):
        _check_pair_against_a(ds, k, gi, gj, rp, cols, s, bbh, alphabet=4)


def test_rejects_letters_outside_the_alphabet():
    ds = synth.from_strings([[b"ACDEFX"], [b"ACDEF"]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.IndexB(ds, 2)
    assert e.value.code == oracle.ERR_ALPHABET
