"""Batched form (pd_bbh_batch): many independent genome-pair jobs, each at its
own k, profiled and compared in a few chunked launch sequences.  Every job's
Best Hits (both directions, with their sum-min) and BBH pairs must equal the
one-pair-per-launch GPU path on that job's two genomes alone, and the oracle
on sampled jobs."""
import os

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


@pytest.fixture(scope="module")
def batch_data():
    # genes per genome U[60, 700] keep the test quick while spanning k = 4..5
    ds, jobs = synth.job_batch(30, seed=4, genes=(60, 700))
    gp = ds.genome_ptr
    n_res = [int(ds.gene_ptr[gp[b + 1]] - ds.gene_ptr[gp[a]]) for a, b in jobs]
    ks = np.array([pd.pd_choose_k(n) for n in n_res], np.int32)
    assert all(oracle.choose_k(n) == k for n, k in zip(n_res, ks))
    return ds, jobs, ks


def _per_job(ds, rp, cols, s, job_ptr, pairs, jobs):
    """Split batch outputs into per-job (bh_ab, s_ab, bh_ba, s_ba, bbh)."""
    gp = ds.genome_ptr
    out, r = [], 0
    for j, (A, B) in enumerate(jobs):
        nA, nB = int(gp[A + 1] - gp[A]), int(gp[B + 1] - gp[B])
        rows = [(cols[rp[x]:rp[x + 1]].tolist(), s[rp[x]:rp[x + 1]].tolist()) for x in range(r, r + nA + nB)]
        r += nA + nB
        bbh = [tuple(p) for p in pairs[job_ptr[j]:job_ptr[j + 1]].tolist()]
        out.append((rows[:nA], rows[nA:], bbh))
    assert r == len(rp) - 1
    return out


def _run_batch(ctx, ds, jobs, ks, **tuning):
    b = pd.pd_bbh_batch(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, jobs, ks, **tuning)
    rp, cols, s = pd.pd_batch_copy_hits(ctx, b)
    job_ptr, pairs = pd.pd_batch_copy_bbh(ctx, b)
    return _per_job(ds, rp, cols, s, job_ptr, pairs, jobs), pd.pd_batch_get_info(b)


def _per_pair(ctx, ds, A, B, k):
    """One job through the one-pair-per-launch path on its two genomes alone."""
    sub = ds.subset([int(A), int(B)])
    prof = pd.pd_build_profiles(ctx, sub.residues, sub.gene_ptr, sub.genome_ptr, int(k))

    def rows(gi, gj):
        rp, c, s = pd.pd_hits_copy(ctx, pd.pd_best_hits(ctx, prof, gi, gj))
        return [(c[rp[x]:rp[x + 1]].tolist(), s[rp[x]:rp[x + 1]].tolist()) for x in range(len(rp) - 1)]

    bbh = [tuple(p) for p in pd.pd_bbh_copy(ctx, pd.pd_bbh(ctx, prof, 0, 1)).tolist()]
    return rows(0, 1), rows(1, 0), bbh


def test_batch_equals_per_pair_path(ctx, batch_data):
    ds, jobs, ks = batch_data
    got, info = _run_batch(ctx, ds, jobs, ks, max_chunk_jobs=7)
    assert info.n_jobs == len(jobs) and info.n_chunks >= 5
    for j, (A, B) in enumerate(jobs):
        assert got[j] == _per_pair(ctx, ds, A, B, ks[j]), f"job {j}"


def test_chunking_does_not_change_results(ctx, batch_data):
    ds, jobs, ks = batch_data
    one, info1 = _run_batch(ctx, ds, jobs, ks)
    many, info2 = _run_batch(ctx, ds, jobs, ks, max_chunk_jobs=3, max_chunk_windows=200_000)
    assert info2.n_chunks > info1.n_chunks
    assert one == many


@pytest.mark.parametrize("j", [0, 7, 19])
def test_sampled_jobs_against_oracle(ctx, batch_data, j):
    ds, jobs, ks = batch_data
    got, _ = _run_batch(ctx, ds, jobs, ks, max_chunk_jobs=7)
    A, B = (int(x) for x in jobs[j])
    sub = ds.subset([A, B])
    R = oracle.pair_for_dataset(sub, 0, 1, int(ks[j]), n_threads=os.cpu_count() or 4)
    ab, ba, bbh = got[j]
    assert [c for c, _ in ab] == [R.row_bh(a).tolist() for a in range(R.S.shape[0])]
    assert [s for _, s in ab] == [[int(R.S[a, b]) for b in R.row_bh(a)] for a in range(R.S.shape[0])]
    assert [c for c, _ in ba] == [R.col_bh(b).tolist() for b in range(R.S.shape[1])]
    assert [s for _, s in ba] == [[int(R.S[a, b]) for a in R.col_bh(b)] for b in range(R.S.shape[1])]
    assert bbh == [tuple(x) for x in R.bbh.tolist()]


def test_mixed_k_and_shared_genomes(ctx, batch_data):
    """Jobs in any genome order (reversed pairs, a genome in several jobs) are
    read in place through per-gene offsets; k differs between jobs."""
    ds, _, _ = batch_data
    jobs = np.array([[1, 0], [3, 0], [5, 4], [0, 5], [9, 2], [2, 9]], np.uint32)
    ks = np.array([3, 4, 5, 4, 6, 3], np.int32)
    got, info = _run_batch(ctx, ds, jobs, ks, max_chunk_jobs=2)
    assert info.n_chunks >= 4
    for j, (A, B) in enumerate(jobs):
        assert got[j] == _per_pair(ctx, ds, A, B, ks[j]), f"job {j}"


def test_empty_batch_and_errors(ctx, batch_data):
    ds, _, _ = batch_data
    got, info = _run_batch(ctx, ds, np.zeros((0, 2), np.uint32), np.zeros(0, np.int32))
    assert got == [] and info.n_jobs == 0 and info.n_hits == 0
    with pytest.raises(pd.PdError) as e:
        pd.pd_bbh_batch(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, np.array([[2, 2]], np.uint32),
                        np.array([5], np.int32))
    assert e.value.status == 1
    with pytest.raises(pd.PdError) as e:
        pd.pd_bbh_batch(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, np.array([[0, 1]], np.uint32),
                        np.array([9], np.int32))
    assert e.value.status == 4


def test_segmented_profiles_match_separate_builds(ctx, batch_data):
    """Two datasets profiled as two segments of one build: each segment's
    multiplicity vectors and all-pairs Best Hits equal its own build."""
    ds, jobs, _ = batch_data
    sub = ds.subset([0, 1, 2, 3])
    k = 4
    seg = np.array([0, 0, 1, 1], np.uint32)
    prof = pd.pd_build_profiles_segmented(ctx, sub.residues, sub.gene_ptr, sub.genome_ptr, seg, k)
    mv_ptr, codes, counts, La = pd.pd_profiles_copy_mv(ctx, prof)
    rp, cols, s = pd.pd_hits_copy(ctx, pd.pd_best_hits_all(ctx, prof))
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, pd.pd_best_hits_all(ctx, prof)))
    gp = sub.genome_ptr
    n_codes = 20 ** k
    for part, genomes in enumerate([[0, 1], [2, 3]]):
        alone = ds.subset(genomes)
        p1 = pd.pd_build_profiles(ctx, alone.residues, alone.gene_ptr, alone.genome_ptr, k)
        m1, c1, n1, L1 = pd.pd_profiles_copy_mv(ctx, p1)
        g0, g1 = int(gp[genomes[0]]), int(gp[genomes[1] + 1])
        e0, e1 = int(mv_ptr[g0]), int(mv_ptr[g1])
        assert np.array_equal(mv_ptr[g0:g1 + 1] - mv_ptr[g0], m1)
        assert np.array_equal(codes[e0:e1] - part * n_codes, c1)
        assert np.array_equal(counts[e0:e1], n1) and np.array_equal(La[g0:g1], L1)
        rp1, c1h, s1 = pd.pd_hits_copy(ctx, pd.pd_best_hits_all(ctx, p1))
        for x in range(g1 - g0):
            assert (cols[rp[g0 + x]:rp[g0 + x + 1]] - g0).tolist() == c1h[rp1[x]:rp1[x + 1]].tolist()
            assert s[rp[g0 + x]:rp[g0 + x + 1]].tolist() == s1[rp1[x]:rp1[x + 1]].tolist()
        b1 = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, p1, pd.pd_best_hits_all(ctx, p1)))
        sel = (bbh[:, 0] >= g0) & (bbh[:, 0] < g1)
        assert (bbh[sel] - g0).tolist() == b1.tolist()


def test_query_order_and_autotuner(ctx, batch_data):
    ds, jobs, ks = batch_data
    a, _ = _run_batch(ctx, ds, jobs, ks, query_order=0)
    b, _ = _run_batch(ctx, ds, jobs, ks, query_order=1, max_chunk_jobs=4)
    assert a == b
    # every posting walk gives the same bytes
    for walk in (pd.PD_WALK_MERGE, pd.PD_WALK_WARP):
        w, _ = _run_batch(ctx, ds, jobs, ks, walk=walk)
        assert w == a, walk
    best, ms = pd.pd_batch_autotune(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, jobs, ks, n_sample=12)
    assert best["query_order"] in (0, 1) and best["max_chunk_jobs"] in (0, 8, 32) and ms > 0
    assert best["walk"] in (pd.PD_WALK_AUTO, pd.PD_WALK_MERGE, pd.PD_WALK_WARP)
    c, _ = _run_batch(ctx, ds, jobs, ks, **best)
    assert c == a
