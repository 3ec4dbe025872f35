"""Pins of the oracle on the nucleotide alphabet (|Gamma| = 4, ACGT): brute
force on tiny random genomes, a hand-worked case, letter checks, and the k
rule's closed forms at base 4."""
import pytest

import oracle
from paper_2510_23679_gb300 import synth
from tests.test_oracle_pins import brute_pair, csr_lists


def _run(rows, cols, k):
    ds = synth.from_strings([rows, cols])
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, k, alphabet=4)
    return oracle.pair(prof, ds.genome_ptr, 0, 1)


def test_hand_worked():
    # k=3: ACGTAC windows ACG CGT GTA TAC; ACGTTT windows ACG CGT GTT TTT
    R = _run([b"ACGTAC"], [b"ACGTTT", b"GGGG"], 3)
    assert R.S.tolist() == [[2, 0]]
    assert R.Den.tolist() == [[6, 6]]  # 4 + 4 - 2, and 4 + 2 - 0
    assert R.row_bh(0).tolist() == [0] and R.bbh.tolist() == [[0, 0]]


@pytest.mark.parametrize("seed", range(8))
def test_brute_force(seed):
    ds = synth.random_tiny(700 + seed, n_genomes=2, max_genes=6, max_len=25, letters=b"ACGT")
    rows = [ds.gene(g) for g in range(ds.genome_ptr[0], ds.genome_ptr[1])]
    cols = [ds.gene(g) for g in range(ds.genome_ptr[1], ds.genome_ptr[2])]
    for k in (1, 2, 4, 6):
        R = _run(rows, cols, k)
        row_bh, col_bh, bbh = brute_pair(rows, cols, k)
        assert csr_lists(R.row_ptr, R.row_col) == row_bh
        assert csr_lists(R.col_ptr, R.col_row) == col_bh
        assert [tuple(x) for x in R.bbh.tolist()] == bbh


def test_letters():
    ds = synth.from_strings([[b"ACGU"], [b"ACG"]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.Profiles(ds.residues, ds.gene_ptr, 2, alphabet=4)
    assert e.value.code == oracle.ERR_ALPHABET
    # an amino-acid letter outside ACGT is rejected at base 4, accepted at base 20
    ds = synth.from_strings([[b"ACDG"], [b"ACG"]])
    with pytest.raises(oracle.OracleError):
        oracle.Profiles(ds.residues, ds.gene_ptr, 2, alphabet=4)
    oracle.Profiles(ds.residues, ds.gene_ptr, 2)


def test_k_rule_base_4():
    for k in range(1, 20):
        assert oracle.choose_k(4 ** k, alphabet=4) == k
        assert oracle.choose_k(4 ** k + 1, alphabet=4) == k + 1
