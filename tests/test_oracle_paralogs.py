"""Pins of the oracle's within-genome Best Hits: a hand-made genome with
known paralogs, and brute force (windows matched one by one, exact
fractions) on tiny random genomes."""
import pytest

import oracle
from paper_2510_23679_gb300 import synth
from tests.test_oracle_pins import brute_bh


def test_hand_made_paralogs():
    # k=2: genes 0 and 1 are identical (GJ 1); gene 2 shares AC, CD with both
    # (s=2, den 4+3-2... computed by hand below); gene 3 shares nothing.
    ds = synth.from_strings([[b"ACDEF", b"ACDEF", b"ACDW", b"YYYY"]])
    rows = oracle.paralog_hits(ds, 2)
    assert [c for c, _ in rows] == [[1], [0], [0, 1], []]
    # gene 2 (AC CD DW) vs 0 (AC CD DE EF): s=2, sum-max = 5; same for gene 1
    assert [s for _, s in rows] == [[4], [4], [2, 2], []]
    assert oracle.paralog_bbh(rows) == [(0, 1)]


@pytest.mark.parametrize("seed", range(6))
def test_brute_force(seed):
    ds = synth.random_tiny(100 + seed, n_genomes=2, max_genes=6, max_len=14, letters=b"ACD")
    k = 2
    rows = oracle.paralog_hits(ds, k)
    gp = ds.genome_ptr
    for i in range(ds.n_genomes):
        genes = [ds.gene(g) for g in range(gp[i], gp[i + 1])]
        for a in range(len(genes)):
            others = [g for b, g in enumerate(genes) if b != a]
            idx = [b for b in range(len(genes)) if b != a]
            exp = [int(gp[i]) + idx[t] for t in brute_bh(genes[a], others, k)]
            assert rows[int(gp[i]) + a][0] == exp
