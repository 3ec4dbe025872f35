"""Nucleotide alphabet (ACGT, base-4 codes, k up to 16) on the GPU against the
oracle: the nt8x600 workload (all ordered genome pairs sampled), tiny random
datasets over k = 1..16, multiplicity vectors, and the alphabet/k checks."""
import os

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


def _decode4(code, k):
    out = bytearray(k)
    for t in range(k - 1, -1, -1):
        out[t] = b"ACGT"[code % 4]
        code //= 4
    return bytes(out)


def _check_pair(ctx, prof, ds, gi, gj, k):
    R = oracle.pair_for_dataset(ds, gi, gj, k, n_threads=os.cpu_count() or 4, alphabet=4)
    h = pd.pd_best_hits(ctx, prof, gi, gj)
    rp, cols, s = pd.pd_hits_copy(ctx, h)
    assert [cols[rp[a]:rp[a + 1]].tolist() for a in range(len(rp) - 1)] == \
        [R.row_bh(a).tolist() for a in range(R.S.shape[0])]
    assert [s[rp[a]:rp[a + 1]].tolist() for a in range(len(rp) - 1)] == \
        [[int(R.S[a, b]) for b in R.row_bh(a)] for a in range(R.S.shape[0])]
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh(ctx, prof, gi, gj))
    assert bbh.tolist() == R.bbh.tolist()


def test_workload_pairs(ctx):
    ds = synth.workload("nt8x600")
    k = pd.pd_choose_k(ds.n_residues, 4)
    assert k == oracle.choose_k(ds.n_residues, alphabet=4) == 12
    prof = pd.pd_build_profiles_alphabet(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 4, k)
    assert pd.pd_profiles_get_info(prof).alphabet == 4
    for gi, gj in [(0, 1), (3, 6), (7, 2)]:
        _check_pair(ctx, prof, ds, gi, gj, k)
    # all-pairs form agrees with the per-pair form on one pair
    rp, cols, s = pd.pd_hits_copy(ctx, pd.pd_best_hits_all(ctx, prof))
    gp = ds.genome_ptr
    h = pd.pd_best_hits(ctx, prof, 0, 1)
    rp1, c1, _ = pd.pd_hits_copy(ctx, h)
    for a in range(int(gp[1])):
        row = cols[rp[a]:rp[a + 1]]
        assert (row[(row >= gp[1]) & (row < gp[2])] - gp[1]).tolist() == c1[rp1[a]:rp1[a + 1]].tolist()


@pytest.mark.parametrize("seed", range(4))
def test_tiny_random_all_k(ctx, seed):
    ds = synth.random_tiny(900 + seed, n_genomes=2, max_genes=6, max_len=40, letters=b"ACGT")
    for k in (1, 2, 3, 5, 8, 11, 16):
        prof = pd.pd_build_profiles_alphabet(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 4, k)
        _check_pair(ctx, prof, ds, 0, 1, k)
        _check_pair(ctx, prof, ds, 1, 0, k)


def test_multiplicity_vectors(ctx):
    ds = synth.random_tiny(950, n_genomes=2, max_genes=5, max_len=60, letters=b"ACGT")
    k = 5
    prof = pd.pd_build_profiles_alphabet(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 4, k)
    mv_ptr, codes, counts, La = pd.pd_profiles_copy_mv(ctx, prof)
    ref = oracle.Profiles(ds.residues, ds.gene_ptr, k, alphabet=4)
    for g in range(ds.n_genes):
        kmers, cnts = ref.mv(g)
        got = [(_decode4(int(c), k), int(n)) for c, n in zip(codes[mv_ptr[g]:mv_ptr[g + 1]],
                                                             counts[mv_ptr[g]:mv_ptr[g + 1]])]
        assert got == list(zip(kmers, cnts))


def test_alphabet_errors(ctx):
    ds = synth.from_strings([[b"ACGTN"], [b"ACGT"]])
    with pytest.raises(pd.PdError) as e:
        pd.pd_build_profiles_alphabet(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 4, 2)
    assert e.value.status == 2
    ok = synth.from_strings([[b"ACGT"], [b"ACGT"]])
    with pytest.raises(pd.PdError) as e:
        pd.pd_build_profiles_alphabet(ctx, ok.residues, ok.gene_ptr, ok.genome_ptr, 4, 17)
    assert e.value.status == 4
    with pytest.raises(pd.PdError) as e:
        pd.pd_build_profiles_alphabet(ctx, ok.residues, ok.gene_ptr, ok.genome_ptr, 5, 2)
    assert e.value.status == 1
