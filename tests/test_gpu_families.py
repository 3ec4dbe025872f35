"""Gene families (pd_components / pd_families) against the oracle: random
and adversarial graphs, and the families of the 4-genome workload's BBH graph."""
import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


def _graphs():
    rng = np.random.default_rng(11)
    out = [("empty", 7, np.zeros(0, np.int32), np.zeros(0, np.int32))]
    n = 100_000
    out.append(("path", n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)))
    out.append(("path_reversed", n, np.arange(n - 1, 0, -1, dtype=np.int32), np.arange(n - 2, -1, -1, dtype=np.int32)))
    out.append(("star", n, np.full(n - 1, n - 1, np.int32), np.arange(n - 1, dtype=np.int32)))
    for i, (nn, m) in enumerate([(10, 5), (1000, 800), (50_000, 60_000), (200_000, 150_000)]):
        out.append((f"random{i}", nn, rng.integers(0, nn, m).astype(np.int32), rng.integers(0, nn, m).astype(np.int32)))
    return out


@pytest.mark.parametrize("name,n,a,b", _graphs(), ids=[g[0] for g in _graphs()])
def test_components_against_oracle(ctx, name, n, a, b):
    lab, nc = pd.pd_components(ctx, a, b, n)
    ref = oracle.families(n, zip(a.tolist(), b.tolist()))
    assert np.array_equal(lab, ref)
    assert nc == len(np.unique(ref))


def test_device_edges_and_bad_ids(ctx):
    import torch
    a = torch.tensor([0, 2, 4], dtype=torch.int32, device="cuda")
    b = torch.tensor([1, 3, 3], dtype=torch.int32, device="cuda")
    lab, nc = pd.pd_components(ctx, a, b, 6)
    assert lab.tolist() == [0, 0, 2, 2, 2, 5] and nc == 3
    with pytest.raises(pd.PdError) as e:
        pd.pd_components(ctx, np.array([0, 9], np.int32), np.array([1, 1], np.int32), 4)
    assert e.value.status == 1


def test_families_of_the_bbh_graph(ctx):
    ds = synth.workload("pan4x250")
    k = pd.pd_choose_k(ds.n_residues)
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    bbh = pd.pd_bbh_all(ctx, prof, pd.pd_best_hits_all(ctx, prof))
    lab, nf = pd.pd_families(ctx, bbh, ds.n_genes)
    ref_pairs = oracle.all_pairs_bbh(ds, k)
    assert pd.pd_bbh_copy(ctx, bbh).tolist() == ref_pairs.tolist()
    ref = oracle.families(ds.n_genes, ref_pairs.tolist())
    assert np.array_equal(lab, ref) and nf == len(np.unique(ref))
