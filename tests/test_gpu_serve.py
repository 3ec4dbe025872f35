"""Served form (pd_index_*): a resident index answers incoming genomes with
their Best Hits in every resident genome and their BBH pairs, then takes them
in.  Each answer must equal the plain path on a dataset made of the
request's snapshot (the genomes resident at submission) plus the request's
genome, whether the request ran alone or together with others."""
import os

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu

N_RES, N_INC = 4, 8
BUDGET = 8 << 30


@pytest.fixture(scope="module")
def ctx():
    return pd.pd_ctx_create(0)


@pytest.fixture(scope="module")
def stream():
    ds = synth.served_stream(N_RES, N_INC, seed=5, resident_genes=("uniform", 200, 400), incoming_genes=(150, 500),
                             n_families=500)
    res = ds.subset(list(range(N_RES)))
    k = pd.pd_choose_k(res.n_residues)
    assert k == oracle.choose_k(res.n_residues)
    return ds, res, k


def _reply(index, ticket):
    r = pd.pd_index_poll(index, ticket, 60_000)
    info = pd.pd_reply_get_info(r)
    rp, cols, s, bbh = pd.pd_reply_copy(r)
    rows = [(cols[rp[x]:rp[x + 1]].tolist(), s[rp[x]:rp[x + 1]].tolist()) for x in range(len(rp) - 1)]
    return info, rows, [tuple(p) for p in bbh.tolist()]


def _expected(ctx, ds, resident_order, x, k):
    """Plain path on (snapshot genomes in resident order) + genome x."""
    sub = ds.subset(list(resident_order) + [x])
    prof = pd.pd_build_profiles(ctx, sub.residues, sub.gene_ptr, sub.genome_ptr, k)
    hits = pd.pd_best_hits_all(ctx, prof)
    rp, cols, s = pd.pd_hits_copy(ctx, hits)
    g0 = int(sub.genome_ptr[-2])
    rows = [(cols[rp[a]:rp[a + 1]].tolist(), s[rp[a]:rp[a + 1]].tolist()) for a in range(g0, sub.n_genes)]
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits))
    pairs = sorted((int(a) - g0, int(b)) for b, a in bbh.tolist() if a >= g0)  # genome(b) < genome(a) = x
    return rows, pairs, sub


def _index(ctx, res, k, budget=BUDGET):
    return pd.pd_index_create(ctx, res.residues, res.gene_ptr, res.genome_ptr, k, budget)


def test_sequential_requests_grow_the_index(ctx, stream):
    ds, res, k = stream
    index = _index(ctx, res, k)
    order = list(range(N_RES))
    for x in range(N_RES, N_RES + N_INC):
        r, gp = synth.genome_of(ds, x)
        t = pd.pd_index_submit(index, r, gp)
        info, rows, bbh = _reply(index, t)
        assert info.status == 0 and info.snapshot_genomes == len(order)
        exp_rows, exp_bbh, _ = _expected(ctx, ds, order, x, k)
        assert rows == exp_rows, f"genome {x}"
        assert bbh == exp_bbh, f"genome {x}"
        order.append(x)
    ii = pd.pd_index_get_info(index)
    assert ii.n_genomes == N_RES + N_INC and ii.requests_done == N_INC
    assert np.array_equal(pd.pd_index_genome_ptr(index, ii.n_genomes),
                          ds.subset(order).genome_ptr)


def test_answer_against_oracle(ctx, stream):
    ds, res, k = stream
    index = _index(ctx, res, k)
    x = N_RES
    r, gp = synth.genome_of(ds, x)
    info, rows, bbh = _reply(index, pd.pd_index_submit(index, r, gp))
    sub = ds.subset(list(range(N_RES)) + [x])
    gptr = sub.genome_ptr
    for j in (0, N_RES - 1):
        R = oracle.pair_for_dataset(sub, N_RES, j, k, n_threads=os.cpu_count() or 4)
        j0, j1 = int(gptr[j]), int(gptr[j + 1])
        for a in range(R.S.shape[0]):
            got = [(c - j0, s) for c, s in zip(*rows[a]) if j0 <= c < j1]
            assert [c for c, _ in got] == R.row_bh(a).tolist()
            assert [s for _, s in got] == [int(R.S[a, b]) for b in R.row_bh(a)]
        assert [(a, b - j0) for a, b in bbh if j0 <= b < j1] == [tuple(p) for p in R.bbh.tolist()]


def test_alone_and_in_a_mix_agree(ctx, stream):
    """The same genome answered alone and inside a burst that provably shares
    one launch sequence: admission is held while the burst is queued, then
    released, so every request of the burst is admitted by the same tick."""
    ds, res, k = stream
    x0 = N_RES
    r, gp = synth.genome_of(ds, x0)
    alone_idx = _index(ctx, res, k)
    alone = _reply(alone_idx, pd.pd_index_submit(alone_idx, r, gp))
    assert alone[0].tick_requests == 1
    mix_idx = _index(ctx, res, k)
    pd.pd_index_hold(mix_idx, True)
    tickets = [pd.pd_index_submit(mix_idx, r, gp)]
    for x in range(N_RES + 1, N_RES + N_INC):
        tickets.append(pd.pd_index_submit(mix_idx, *synth.genome_of(ds, x)))
    assert pd.pd_index_get_info(mix_idx).queued == N_INC
    pd.pd_index_hold(mix_idx, False)
    replies = [_reply(mix_idx, t) for t in tickets]
    info0 = replies[0][0]
    assert info0.snapshot_genomes == N_RES
    assert info0.tick_requests == N_INC, "the checked request did not share its tick with the burst"
    assert all(rep[0].t_start_ns == info0.t_start_ns for rep in replies), "the burst ran in more than one tick"
    assert replies[0][1:] == alone[1:]
    # every other answer equals the plain path at its own snapshot (all of the
    # burst was submitted before any of it was answered: snapshot = N_RES)
    for (info, rows, bbh), x in zip(replies, range(N_RES, N_RES + N_INC)):
        assert info.snapshot_genomes == N_RES
        exp_rows, exp_bbh, _ = _expected(ctx, ds, list(range(N_RES)), x, k)
        assert rows == exp_rows and bbh == exp_bbh, f"genome {x}"
    ii = pd.pd_index_get_info(mix_idx)
    assert ii.requests_done == N_INC and ii.max_tick_requests == N_INC and ii.ticks == 1


def test_poll_times_out_on_a_pending_request(ctx, stream):
    ds, res, k = stream
    index = _index(ctx, res, k)
    pd.pd_index_hold(index, True)
    t = pd.pd_index_submit(index, *synth.genome_of(ds, N_RES))
    for wait_ms in (0, 50):
        with pytest.raises(pd.PdError) as e:
            pd.pd_index_poll(index, t, wait_ms)
        assert e.value.status == 8  # PD_ERR_TIMEOUT
    pd.pd_index_hold(index, False)
    info, rows, bbh = _reply(index, t)
    assert info.status == 0 and len(rows) == int(np.diff(synth.genome_of(ds, N_RES)[1]).size)
    with pytest.raises(pd.PdError) as e:  # each answer is returned once
        pd.pd_index_poll(index, t, 0)
    assert e.value.status == 8


def test_budget_and_arguments(ctx, stream):
    ds, res, k = stream
    with pytest.raises(pd.PdError) as e:
        _index(ctx, res, k, budget=1 << 20)
    assert e.value.status == 6
    index = _index(ctx, res, k, budget=2 << 30)
    big = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY" * 40_000_000, np.uint8)
    with pytest.raises(pd.PdError) as e:
        pd.pd_index_submit(index, big, np.array([0, 2_000, big.size], np.int64))
    assert e.value.status in (3, 6)  # a gene too long, or over the budget
    with pytest.raises(pd.PdError) as e:
        pd.pd_index_poll(index, 12345, 0)
    assert e.value.status == 1
    with pytest.raises(pd.PdError) as e:
        pd.pd_index_submit(index, np.frombuffer(b"ACDEFGXB", np.uint8), np.array([0, 8], np.int64))
    assert e.value.status == 2


def test_many_arrivals_cross_level_merges(ctx, stream):
    """A longer stream, submitted in bursts: the delta level is rebuilt and
    merged into the base several times; every answer still equals the plain
    path at its snapshot."""
    ds, res, k = stream
    big = synth.served_stream(N_RES, 24, seed=9, resident_genes=("uniform", 200, 400), incoming_genes=(150, 500),
                              n_families=500)
    res = big.subset(list(range(N_RES)))
    index = _index(ctx, res, k)
    commit_order = list(range(big.n_genomes))  # answers commit in submission order
    x = N_RES
    while x < big.n_genomes:
        burst = list(range(x, min(x + 5, big.n_genomes)))
        tickets = [pd.pd_index_submit(index, *synth.genome_of(big, g)) for g in burst]
        for t, g in zip(tickets, burst):
            info, rows, bbh = _reply(index, t)
            assert N_RES <= info.snapshot_genomes <= g
            exp_rows, exp_bbh, _ = _expected(ctx, big, commit_order[:info.snapshot_genomes], g, k)
            assert rows == exp_rows and bbh == exp_bbh, f"genome {g}"
        x += len(burst)
    assert pd.pd_index_get_info(index).n_genomes == big.n_genomes
