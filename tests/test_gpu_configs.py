"""Parity at the stated shapes of the batched and served workloads, against
oracle B (pd_oracle_b.c, pinned to oracle A in test_oracle_b.py).

* Batched form: ``synth.job_batch(2000, seed=4)`` -- 2000 genome-pair jobs,
  gene counts U[500, 6000], half of the jobs with median gene length 300 aa
  and half 900 aa, each at its own k -- through ``pd_bbh_batch``.  Every job's
  Best Hit CSR (both directions, with sum-min) and BBH pairs equal the
  one-pair-per-launch GPU path on its two genomes; a seeded sample of the
  jobs equals oracle B element by element.
* Served form: a resident index of 100 genomes of the pan50x3000 model; the
  first 24 incoming genomes (U[1000, 7000] genes) are submitted in bursts of
  four (admission held while a burst is queued, so each burst shares its
  launches); every answer -- Best Hits in every resident genome of its
  snapshot, with sum-min, and its BBH pairs -- equals oracle B computed over
  the snapshot's genomes.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu

N_JOBS = 2000
ORACLE_JOBS = 200


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


def _job_view(rp, cols, s, nA, nB):
    """A two-genome dataset's all-pairs CSR (global ids, genome A first) in the
    batch layout: A's rows with columns local to B, then B's rows with
    columns local to A."""
    r = rp - rp[0]
    c = cols[rp[0]:rp[-1]].astype(np.int64).copy()
    c[:r[nA]] -= nA
    return r, c, s[rp[0]:rp[-1]]


def _bbh_view(pairs, nA):
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2).copy()
    p[:, 1] -= nA
    return p


@pytest.fixture(scope="module")
def job_batch():
    ds, jobs = synth.job_batch(N_JOBS, seed=4, workers=oracle.default_threads())
    gp = ds.genome_ptr
    n_res = [int(ds.gene_ptr[gp[b + 1]] - ds.gene_ptr[gp[a]]) for a, b in jobs]
    ks = np.array([pd.pd_choose_k(n) for n in n_res], np.int32)
    return ds, jobs, ks


@pytest.fixture(scope="module")
def batch_result(ctx, job_batch):
    ds, jobs, ks = job_batch
    b = pd.pd_bbh_batch(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, jobs, ks)
    rp, cols, s = pd.pd_batch_copy_hits(ctx, b)
    job_ptr, pairs = pd.pd_batch_copy_bbh(ctx, b)
    info = pd.pd_batch_get_info(b)
    gp = ds.genome_ptr
    per_job, r = [], 0
    for j, (A, B) in enumerate(jobs):
        nA, nB = int(gp[A + 1] - gp[A]), int(gp[B + 1] - gp[B])
        sl = rp[r:r + nA + nB + 1]
        per_job.append((nA, nB, sl - sl[0], cols[sl[0]:sl[-1]].astype(np.int64), s[sl[0]:sl[-1]],
                        pairs[job_ptr[j]:job_ptr[j + 1]].astype(np.int64)))
        r += nA + nB
    assert r == len(rp) - 1 and info.n_jobs == N_JOBS
    return per_job, info


def test_batch_at_stated_shape_equals_one_pair_path(ctx, job_batch, batch_result):
    import torch
    ds, jobs, ks = job_batch
    per_job, info = batch_result
    sizes = np.diff(ds.genome_ptr)
    assert sizes.min() >= 500 and sizes.max() <= 6000
    dev = torch.device("cuda", 0)
    res_d = torch.from_numpy(ds.residues).to(dev)
    gp_d = torch.from_numpy(ds.gene_ptr).to(dev)
    n_hits = n_bbh = 0
    for j, (A, B) in enumerate(jobs):
        nA, nB, rp, cols, s, bbh = per_job[j]
        g0, g1 = int(ds.genome_ptr[A]), int(ds.genome_ptr[A + 1])
        h0, h1 = int(ds.genome_ptr[B]), int(ds.genome_ptr[B + 1])
        assert g1 == h0, "jobs hold adjacent genomes"
        r0, r1 = int(ds.gene_ptr[g0]), int(ds.gene_ptr[h1])
        prof = pd.pd_build_profiles(ctx, res_d[r0:r1], (gp_d[g0:h1 + 1] - r0).contiguous(),
                                    np.array([0, nA, nA + nB], np.int32), int(ks[j]))
        hits = pd.pd_best_hits_all(ctx, prof)
        wrp, wcols, ws = _job_view(*pd.pd_hits_copy(ctx, hits), nA, nB)
        wbbh = _bbh_view(pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits)), nA)
        assert np.array_equal(rp, wrp) and np.array_equal(cols, wcols) and np.array_equal(s, ws), f"job {j}"
        assert np.array_equal(bbh, wbbh), f"job {j}"
        n_hits += len(cols)
        n_bbh += len(bbh)
    assert n_hits == info.n_hits and n_bbh == info.n_bbh


def test_batch_at_stated_shape_equals_oracle_b(job_batch, batch_result):
    ds, jobs, ks = job_batch
    per_job, _ = batch_result
    rng = np.random.default_rng(44)
    sample = sorted(rng.choice(N_JOBS, ORACLE_JOBS, replace=False).tolist())

    def expected(j):
        A, B = (int(x) for x in jobs[j])
        sub = ds.subset([A, B])
        assert oracle.choose_k(sub.n_residues) == int(ks[j])
        rp, cols, s, bbh = oracle.all_pairs_b(oracle.IndexB(sub, int(ks[j]), n_threads=1))
        nA = int(sub.genome_ptr[1])
        return _job_view(rp, cols, s, nA, sub.n_genes - nA), _bbh_view(bbh, nA)

    with ThreadPoolExecutor(oracle.default_threads()) as ex:
        for j, ((wrp, wcols, ws), wbbh) in zip(sample, ex.map(expected, sample)):
            nA, nB, rp, cols, s, bbh = per_job[j]
            assert np.array_equal(rp, wrp) and np.array_equal(cols, wcols), f"job {j}: Best Hits"
            assert np.array_equal(s, ws), f"job {j}: sum-min"
            assert np.array_equal(bbh, wbbh), f"job {j}: BBH"


N_RESIDENT, N_REQUESTS, BURST = 100, 24, 4


def test_served_at_stated_shape_equals_oracle_b(ctx):
    ds = synth.served_stream(N_RESIDENT, N_REQUESTS, seed=5)
    res = ds.subset(list(range(N_RESIDENT)))
    k = pd.pd_choose_k(res.n_residues)
    assert k == oracle.choose_k(res.n_residues)
    index = pd.pd_index_create(ctx, res.residues, res.gene_ptr, res.genome_ptr, k, 120 << 30)
    idx = oracle.IndexB(ds, k)  # every genome; each answer's targets are its snapshot
    gp = ds.genome_ptr
    checked = 0
    for x0 in range(N_RESIDENT, ds.n_genomes, BURST):
        burst = list(range(x0, min(x0 + BURST, ds.n_genomes)))
        pd.pd_index_hold(index, True)
        tickets = [pd.pd_index_submit(index, *synth.genome_of(ds, x)) for x in burst]
        pd.pd_index_hold(index, False)
        for t, x in zip(tickets, burst):
            rep = pd.pd_index_poll(index, t, 600_000)
            info = pd.pd_reply_get_info(rep)
            assert info.status == 0 and info.snapshot_genomes == x0 and info.tick_requests == len(burst)
            rp, cols, s, bbh = pd.pd_reply_copy(rep)
            genes = np.arange(int(gp[x]), int(gp[x + 1]), dtype=np.uint32)
            wrp, wcols, ws = oracle.best_hits_b(idx, genes, targets=range(x0))
            assert np.array_equal(rp, wrp), f"genome {x}: row lengths"
            assert np.array_equal(cols, wcols) and np.array_equal(s, ws), f"genome {x}: Best Hits"
            # BBH: b a Best Hit of a, and a a Best Hit of b in genome x
            cand = np.unique(wcols).astype(np.uint32)
            brp, bcols, _ = oracle.best_hits_b(idx, cand, targets=[x])
            back = {int(b): set(bcols[brp[i]:brp[i + 1]].tolist()) for i, b in enumerate(cand)}
            want = [(a, int(b)) for a in range(len(genes)) for b in wcols[wrp[a]:wrp[a + 1]]
                    if int(genes[a]) in back[int(b)]]
            assert [tuple(p) for p in bbh.tolist()] == want, f"genome {x}: BBH"
            checked += 1
    assert checked == N_REQUESTS
    assert pd.pd_index_get_info(index).max_tick_requests == BURST
