"""Checks shared by the full-size parity tests (test infrastructure).

A workload is profiled and compared all-against-all on the GPU exactly as
bench.py times it (device-resident inputs, pd_build_profiles,
pd_best_hits_all, pd_bbh_all).  Oracle B (inverted index on host threads,
pinned to oracle A) then recomputes the whole result, every genome pair;
oracle A recomputes sampled genome pairs in full; and properties that hold at
any size are checked on the whole result.
"""
import os

import numpy as np

import oracle
from paper_2510_23679_gb300 import pd, synth


def run_full(name, expect_k):
    import torch
    ds = synth.workload(name)
    k = pd.pd_choose_k(ds.n_residues)
    assert k == oracle.choose_k(ds.n_residues) == expect_k
    ctx = pd.pd_ctx_create(0)
    dev = torch.device("cuda", 0)
    res = torch.from_numpy(ds.residues).to(dev)
    gp = torch.from_numpy(ds.gene_ptr).to(dev)
    gn = torch.from_numpy(ds.genome_ptr).to(dev)
    prof = pd.pd_build_profiles(ctx, res, gp, gn, k)
    hits = pd.pd_best_hits_all(ctx, prof)
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits))
    rp, cols, s = pd.pd_hits_copy(ctx, hits)
    _, _, _, La = pd.pd_profiles_copy_mv(ctx, prof)
    info = pd.pd_hits_get_info(hits)
    del hits, res, gp, gn
    return dict(ds=ds, k=k, ctx=ctx, prof=prof, rp=rp, cols=cols, s=s, bbh=bbh, La=La, info=info)


def check_whole_against_oracle_b(full):
    """Every Best Hit (with its sum-min) of every gene in every other genome,
    and every BBH pair of every genome pair, equal oracle B's."""
    ds = full["ds"]
    idx = oracle.IndexB(ds, full["k"])
    rp, cols, s, bbh = oracle.all_pairs_b(idx)
    del idx
    assert np.array_equal(full["rp"], rp), "Best Hit row lengths"
    assert np.array_equal(full["cols"], cols), "Best Hit columns"
    assert np.array_equal(full["s"], s), "Best Hit sum-min values"
    assert np.array_equal(full["bbh"], bbh), "BBH pairs"


def rows_towards(full, genome_from, genome_to):
    ds, rp, cols, s = full["ds"], full["rp"], full["cols"], full["s"]
    gp = ds.genome_ptr
    t0, t1 = int(gp[genome_to]), int(gp[genome_to + 1])
    out_c, out_s = [], []
    for a in range(int(gp[genome_from]), int(gp[genome_from + 1])):
        row = cols[rp[a]:rp[a + 1]]
        sel = (row >= t0) & (row < t1)
        out_c.append((row[sel] - t0).tolist())
        out_s.append(s[rp[a]:rp[a + 1]][sel].tolist())
    return out_c, out_s


def check_sampled_pair(full, gi, gj):
    """Every Best Hit of both directions and every BBH pair of (gi, gj)."""
    ds = full["ds"]
    R = oracle.pair_for_dataset(ds, gi, gj, full["k"], n_threads=os.cpu_count() or 4)
    rows, svals = rows_towards(full, gi, gj)
    assert rows == [R.row_bh(a).tolist() for a in range(R.S.shape[0])]
    for a, (cs, ss) in enumerate(zip(rows, svals)):
        assert ss == [int(R.S[a, b]) for b in cs]
    cols_, _ = rows_towards(full, gj, gi)
    assert cols_ == [R.col_bh(b).tolist() for b in range(R.S.shape[1])]
    gp = ds.genome_ptr
    a0, b0 = int(gp[gi]), int(gp[gj])
    got = full["bbh"]
    sel = (got[:, 0] >= a0) & (got[:, 0] < int(gp[gi + 1])) & (got[:, 1] >= b0) & (got[:, 1] < int(gp[gj + 1]))
    assert [tuple(x) for x in (got[sel] - [a0, b0]).tolist()] == [tuple(x) for x in R.bbh.tolist()]
    # the one-pair-per-launch form agrees too
    assert [tuple(x) for x in pd.pd_bbh_copy(full["ctx"], pd.pd_bbh(full["ctx"], full["prof"], gi, gj)).tolist()] == \
        [tuple(x) for x in R.bbh.tolist()]


def check_properties(full):
    ds, rp, cols, s, bbh, La = full["ds"], full["rp"], full["cols"], full["s"], full["bbh"], full["La"]
    gp = ds.genome_ptr.astype(np.int64)
    genome_of = np.repeat(np.arange(ds.n_genomes, dtype=np.int32), np.diff(gp))
    row_of = np.repeat(np.arange(ds.n_genes, dtype=np.int64), np.diff(rp))
    assert len(rp) == ds.n_genes + 1 and rp[-1] == len(cols) == full["info"].n_hits
    # no hit inside the query's own genome; 1 <= s <= min(La, Lb)
    assert np.all(genome_of[cols] != genome_of[row_of])
    assert np.all(s >= 1) and np.all(s <= np.minimum(La[row_of], La[cols]))
    # rows strictly ascending
    same_row = row_of[1:] == row_of[:-1]
    assert np.all(cols[1:][same_row] > cols[:-1][same_row])
    # all hits of a row towards one genome share one ratio s / (La + Lb - s)
    den = La[row_of].astype(np.int64) + La[cols] - s
    key = row_of * ds.n_genomes + genome_of[cols]
    same = key[1:] == key[:-1]
    assert np.all((s[1:].astype(np.int64) * den[:-1])[same] == (s[:-1].astype(np.int64) * den[1:])[same])
    del den, key, same, same_row
    # BBH: ordered, genome(a) < genome(b), and a mutual Best Hit
    assert np.all(genome_of[bbh[:, 0]] < genome_of[bbh[:, 1]])
    order = bbh[:, 0].astype(np.int64) * ds.n_genes + bbh[:, 1]
    assert np.all(np.diff(order) > 0)
    G = np.int64(ds.n_genes)
    fwd = row_of * G + cols  # already sorted: rows ascending, columns ascending in a row
    assert np.all(np.diff(fwd) > 0)
    assert np.all(_in_sorted(bbh[:, 0].astype(np.int64) * G + bbh[:, 1], fwd))
    assert np.all(_in_sorted(bbh[:, 1].astype(np.int64) * G + bbh[:, 0], fwd))
    # every mutual pair of Best Hits is reported
    rev = cols.astype(np.int64) * G + row_of
    mutual = (genome_of[row_of] < genome_of[cols]) & _in_sorted(rev, fwd)
    assert int(mutual.sum()) == len(bbh)


def _in_sorted(q, sorted_keys):
    """Membership of each q in a sorted key array."""
    if len(sorted_keys) == 0:
        return np.zeros(len(q), dtype=bool)
    i = np.minimum(np.searchsorted(sorted_keys, q), len(sorted_keys) - 1)
    return sorted_keys[i] == q
