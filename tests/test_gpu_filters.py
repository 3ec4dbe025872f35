"""Candidate filters theta (Eq. (6)) and tau (Eq. (7)) on the GPU against the
oracle: every ordered genome pair of the 4-genome workload under several
settings (all-pairs and per-pair forms, with BBH), tiny random datasets,
queries forced onto the global-memory tier, and argument checks."""
import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu

SETTINGS = [((0, 1), (0, 1)), ((4, 5), (0, 1)), ((0, 1), (1, 2)), ((3, 5), (1, 3)), ((9, 10), (3, 4))]


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


@pytest.fixture(scope="module")
def pan4(ctx):
    ds = synth.workload("pan4x250")
    k = pd.pd_choose_k(ds.n_residues)
    return ds, k, pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)


def _local_rows(rp, cols, rows, t0, t1):
    out = []
    for a in rows:
        r = cols[rp[a]:rp[a + 1]]
        out.append((r[(r >= t0) & (r < t1)] - t0).tolist())
    return out


@pytest.mark.parametrize("theta,tau", SETTINGS)
def test_workload_against_oracle(ctx, pan4, theta, tau):
    ds, k, prof = pan4
    gp = ds.genome_ptr
    hits = pd.pd_best_hits_all_filtered(ctx, prof, theta, tau)
    rp, cols, _ = pd.pd_hits_copy(ctx, hits)
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits))
    for gi in range(ds.n_genomes):
        for gj in range(gi + 1, ds.n_genomes):
            rows_ref, cols_ref, bbh_ref = oracle.filtered_pair(ds, gi, gj, k, theta, tau)
            assert _local_rows(rp, cols, range(gp[gi], gp[gi + 1]), gp[gj], gp[gj + 1]) == rows_ref
            assert _local_rows(rp, cols, range(gp[gj], gp[gj + 1]), gp[gi], gp[gi + 1]) == cols_ref
            sel = (bbh[:, 0] >= gp[gi]) & (bbh[:, 0] < gp[gi + 1]) & (bbh[:, 1] >= gp[gj]) & (bbh[:, 1] < gp[gj + 1])
            assert [tuple(x) for x in (bbh[sel] - [gp[gi], gp[gj]]).tolist()] == bbh_ref
            # per-pair form
            rp1, c1, _ = pd.pd_hits_copy(ctx, pd.pd_best_hits_filtered(ctx, prof, gi, gj, theta, tau))
            assert [c1[rp1[a]:rp1[a + 1]].tolist() for a in range(len(rp1) - 1)] == rows_ref


@pytest.mark.parametrize("seed", range(4))
def test_tiny_random(ctx, seed):
    ds = synth.random_tiny(600 + seed, n_genomes=2, max_genes=8, max_len=30, letters=b"ACDEG")
    for k in (1, 2, 3):
        prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
        for theta, tau in SETTINGS:
            rows_ref, _, _ = oracle.filtered_pair(ds, 0, 1, k, theta, tau)
            rp, c, _ = pd.pd_hits_copy(ctx, pd.pd_best_hits_filtered(ctx, prof, 0, 1, theta, tau))
            assert [c[rp[a]:rp[a + 1]].tolist() for a in range(len(rp) - 1)] == rows_ref, (k, theta, tau)


def test_global_tier(ctx):
    """5000 identical target genes overflow the shared-memory table: the
    filtered query finishes on the global-memory tier with the same answer."""
    q = b"ACDEFGHIKLMNPQRSTVWYACDEFGHIKL"
    tgt = [q] * 5000 + [q[:20], q[5:]]
    ds = synth.from_strings([[q], tgt])
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 3)
    for theta, tau in [((0, 1), (0, 1)), ((9, 10), (1, 2))]:
        rows_ref, _, _ = oracle.filtered_pair(ds, 0, 1, 3, theta, tau)
        h = pd.pd_best_hits_filtered(ctx, prof, 0, 1, theta, tau)
        rp, c, _ = pd.pd_hits_copy(ctx, h)
        assert [c[rp[a]:rp[a + 1]].tolist() for a in range(len(rp) - 1)] == rows_ref
        assert pd.pd_hits_get_info(h).n_deferred == 0  # deferred straight past tier 2 (counted in def2)


def test_bad_fractions(ctx, pan4):
    _, _, prof = pan4
    for theta, tau in [((2, 1), (0, 1)), ((0, 0), (0, 1)), ((0, 1), (3, 2))]:
        with pytest.raises(pd.PdError) as e:
            pd.pd_best_hits_all_filtered(ctx, prof, theta, tau)
        assert e.value.status == 1
