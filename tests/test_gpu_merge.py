"""pd_summin_list: sum-min and sum-max (Eq. (5)) of listed gene pairs by the
paper's own two-pointer form (merging the two sorted multiplicity vectors,
Algorithm 2).  Every value equals the oracle's, and the scatter path's for
every pair of a genome pair, including pairs that share nothing."""
import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


def _oracle_sums(ds, k, a, b, alphabet=20):
    P = oracle.Profiles(ds.residues, ds.gene_ptr, k, alphabet)
    return np.array([P.summin(int(x), int(y)) for x, y in zip(a, b)], np.int64).reshape(-1, 2)


def test_random_pairs_equal_the_oracle(ctx):
    ds = synth.workload("pan4x250")
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    rng = np.random.default_rng(7)
    a = rng.integers(0, ds.n_genes, 3000).astype(np.uint32)
    b = rng.integers(0, ds.n_genes, 3000).astype(np.uint32)
    a[:20] = b[:20]  # a gene with itself: s = La, den = La
    s, den = pd.pd_summin_list(ctx, prof, a, b)
    want = _oracle_sums(ds, 5, a, b)
    assert np.array_equal(s.astype(np.int64), want[:, 0])
    assert np.array_equal(den.astype(np.int64), want[:, 1])


def test_every_pair_of_a_genome_pair_equals_the_scatter_path(ctx):
    import torch
    ds = synth.workload("pan4x250")
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    gp = ds.genome_ptr
    A = np.arange(gp[1], gp[2], dtype=np.uint32)
    B = np.arange(gp[3], gp[4], dtype=np.uint32)
    a, b = np.repeat(A, len(B)), np.tile(B, len(A))
    dev = torch.device("cuda", 0)
    s_d = torch.zeros(len(a), dtype=torch.int32, device=dev)
    den_d = torch.zeros(len(a), dtype=torch.int32, device=dev)
    pd.pd_summin_list(ctx, prof, torch.from_numpy(a.view(np.int32)).to(dev),
                      torch.from_numpy(b.view(np.int32)).to(dev), s_d, den_d)
    s = s_d.cpu().numpy().astype(np.uint32).reshape(len(A), len(B))
    ta, tb, ts = pd.pd_summin_pairs(ctx, prof, 1, 3)  # the nonzero triples of the scatter path
    want = np.zeros_like(s)
    want[ta, tb] = ts
    assert np.array_equal(s, want)
    _, _, _, La = pd.pd_profiles_copy_mv(ctx, prof)
    den = den_d.cpu().numpy().astype(np.int64).reshape(len(A), len(B))
    assert np.array_equal(den, La[A][:, None].astype(np.int64) + La[B][None, :] - s)


def test_long_vectors_and_edge_cases(ctx):
    """Vectors longer than the shared-memory sort (nucleotide genes of 20k
    distinct k-mers), genes shorter than k, and an empty list."""
    rng = np.random.default_rng(3)
    letters = np.frombuffer(b"ACGT", np.uint8)
    long1 = rng.choice(letters, 20000).tobytes()
    long2 = long1[:9000] + rng.choice(letters, 11000).tobytes()
    ds = synth.from_strings([[long1, b"ACG", b"ACGTACGTACGTA"], [long2, b"", b"ACGTACGTACGTA"]])
    k = 12
    prof = pd.pd_build_profiles_alphabet(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 4, k)
    a = np.array([0, 0, 1, 2, 1, 4, 3], np.uint32)
    b = np.array([3, 0, 4, 5, 1, 4, 0], np.uint32)
    s, den = pd.pd_summin_list(ctx, prof, a, b)
    want = _oracle_sums(ds, k, a, b, alphabet=4)
    assert np.array_equal(s.astype(np.int64), want[:, 0])
    assert np.array_equal(den.astype(np.int64), want[:, 1])
    assert s[0] >= 8900  # the shared prefix
    e, d = pd.pd_summin_list(ctx, prof, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert len(e) == 0 and len(d) == 0
    with pytest.raises(pd.PdError) as err:
        pd.pd_summin_list(ctx, prof, np.array([0], np.uint32), np.array([ds.n_genes], np.uint32))
    assert err.value.status == 1
