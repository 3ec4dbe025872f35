"""Within-genome (paralog) Best Hits and their mutual pairs against the
oracle: the 4-genome workload (which holds paralog copies) and tiny random
datasets."""
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


def _gpu(ctx, ds, k):
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    h = pd.pd_paralog_hits(ctx, prof)
    rp, cols, s = pd.pd_hits_copy(ctx, h)
    rows = [(cols[rp[x]:rp[x + 1]].tolist(), s[rp[x]:rp[x + 1]].tolist()) for x in range(ds.n_genes)]
    bbh = [tuple(p) for p in pd.pd_bbh_copy(ctx, pd.pd_paralog_bbh(ctx, prof, h)).tolist()]
    return rows, bbh


def test_workload_paralogs(ctx):
    ds = synth.workload("pan4x250")
    k = pd.pd_choose_k(ds.n_residues)
    rows, bbh = _gpu(ctx, ds, k)
    ref = oracle.paralog_hits(ds, k)
    assert rows == [(c, s) for c, s in ref]
    assert bbh == oracle.paralog_bbh(ref)
    assert sum(len(c) for c, _ in rows) > 0


@pytest.mark.parametrize("seed", range(5))
def test_tiny_random(ctx, seed):
    ds = synth.random_tiny(300 + seed, n_genomes=3, max_genes=8, max_len=30, letters=b"ACDEG")
    for k in (1, 2, 3):
        rows, bbh = _gpu(ctx, ds, k)
        ref = oracle.paralog_hits(ds, k)
        assert rows == [(c, s) for c, s in ref], (seed, k)
        assert bbh == oracle.paralog_bbh(ref)


def test_cross_genome_bbh_rejects_paralog_hits(ctx):
    ds = synth.workload("pan4x250")
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    with pytest.raises(pd.PdError):
        pd.pd_bbh_all(ctx, prof, pd.pd_paralog_hits(ctx, prof))
