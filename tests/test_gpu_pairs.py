"""pd_bbh_pairs: many genome pairs of one profiled dataset in one launch
sequence.  Every job equals the one-pair calls on the same profiles
(pd_best_hits both ways, pd_bbh), which the other tests tie to the oracle;
one job is also checked against the oracle directly."""
import os

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


def _split(ds, b, jobs):
    rp, cols, s = pd.pd_batch_copy_hits(b.ctx, b)
    job_ptr, pairs = pd.pd_batch_copy_bbh(b.ctx, b)
    gp = ds.genome_ptr
    out, r = [], 0
    for j, (A, B) in enumerate(jobs):
        nA, nB = int(gp[A + 1] - gp[A]), int(gp[B + 1] - gp[B])
        rows = [(cols[rp[x]:rp[x + 1]].tolist(), s[rp[x]:rp[x + 1]].tolist()) for x in range(r, r + nA + nB)]
        r += nA + nB
        out.append((rows[:nA], rows[nA:], [tuple(p) for p in pairs[job_ptr[j]:job_ptr[j + 1]].tolist()]))
    return out


def _one(ctx, prof, A, B):
    def rows(gi, gj):
        rp, c, s = pd.pd_hits_copy(ctx, pd.pd_best_hits(ctx, prof, int(gi), int(gj)))
        return [(c[rp[x]:rp[x + 1]].tolist(), s[rp[x]:rp[x + 1]].tolist()) for x in range(len(rp) - 1)]
    return rows(A, B), rows(B, A), [tuple(p) for p in pd.pd_bbh_copy(ctx, pd.pd_bbh(ctx, prof, int(A), int(B))).tolist()]


def test_every_ordered_pair_of_the_small_workload(ctx):
    ds = synth.workload("pan4x250")
    k = pd.pd_choose_k(ds.n_residues)
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    jobs = np.array([(a, b) for a in range(4) for b in range(4) if a != b] + [(0, 1), (2, 0)], np.uint32)
    got = _split(ds, pd.pd_bbh_pairs(ctx, prof, jobs), jobs)
    for j, (A, B) in enumerate(jobs):
        assert got[j] == _one(ctx, prof, A, B), f"job {j}"
    R = oracle.pair_for_dataset(ds, 2, 3, k)
    ab, _, bbh = got[[tuple(x) for x in jobs.tolist()].index((2, 3))]
    assert [c for c, _ in ab] == [R.row_bh(a).tolist() for a in range(R.S.shape[0])]
    assert bbh == [tuple(x) for x in R.bbh.tolist()]


def test_sampled_pairs_of_the_benchmark_workload(ctx):
    ds = synth.workload("pan50x3000")
    k = pd.pd_choose_k(ds.n_residues)
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    rng = np.random.default_rng(3)
    jobs = []
    while len(jobs) < 200:
        a, b = rng.integers(0, ds.n_genomes, size=2)
        if a != b:
            jobs.append((a, b))
    jobs = np.array(jobs, np.uint32)
    bt = pd.pd_bbh_pairs(ctx, prof, jobs)
    assert pd.pd_batch_get_info(bt).n_jobs == 200
    got = _split(ds, bt, jobs)
    for j in (0, 57, 133, 199):
        assert got[j] == _one(ctx, prof, *jobs[j]), f"job {j}"
    A, B = (int(x) for x in jobs[57])
    R = oracle.pair_for_dataset(ds, A, B, k, n_threads=os.cpu_count() or 4)
    assert got[57][2] == [tuple(x) for x in R.bbh.tolist()]


def test_empty_and_bad_jobs(ctx):
    ds = synth.workload("pan4x250")
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    info = pd.pd_batch_get_info(pd.pd_bbh_pairs(ctx, prof, np.zeros((0, 2), np.uint32)))
    assert info.n_jobs == 0 and info.n_hits == 0 and info.n_bbh == 0
    for bad in ([[1, 1]], [[0, 4]]):
        with pytest.raises(pd.PdError) as e:
            pd.pd_bbh_pairs(ctx, prof, np.array(bad, np.uint32))
        assert e.value.status == 1
