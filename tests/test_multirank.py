"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).  Each rank
profiles its own replica dataset (no data-path collective), the job's rate is
the units of all ranks over the slowest rank's time, and the union of the
ranks' results is what each rank computes alone (checked with the oracle on
one genome pair per rank)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_info()
    ds = bench.make_workload("pan4x250", r)
    k = oracle.choose_k(ds.n_residues)
    R = oracle.pair_for_dataset(ds, 0, 1, k)
    local_s = 0.5 + rank  # a rank-dependent "time"
    rate = bench.whole_job_rate(ds.logical_pairs(), local_s, w)
    slowest = bench.max_over_ranks(local_s, w)
    total = bench.sum_over_ranks(ds.logical_pairs(), w)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), residues=ds.residues, bbh=R.bbh, rate=rate, slowest=slowest,
             total=total, pairs=ds.logical_pairs(), seed=ds.params["seed"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_replicas(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{i}.npz") for i in range(world)]
    # replicas: different seeded datasets
    assert int(r[0]["seed"]) != int(r[1]["seed"])
    assert not np.array_equal(r[0]["residues"], r[1]["residues"])
    # the reductions agree on every rank and follow the definitions
    total = int(r[0]["pairs"]) + int(r[1]["pairs"])
    for x in r:
        assert float(x["slowest"]) == 1.5
        assert int(x["total"]) == total
        assert float(x["rate"]) == pytest.approx(total / 1.5)
    # each rank's result is its own dataset's (rank 0's equals a fresh single-rank run)
    import bench
    import oracle
    ds0 = bench.make_workload("pan4x250", 0)
    R = oracle.pair_for_dataset(ds0, 0, 1, oracle.choose_k(ds0.n_residues))
    assert np.array_equal(r[0]["bbh"], R.bbh)


def _shard_rank_main(rank, world, port, out_dir):
    """One dataset split by query genes: rank r computes the Best Hit rows of
    every world-th gene (oracle B), the pieces are gathered to rank 0 by the
    library's host code (shards.gather_pieces, over gloo)."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    from paper_2510_23679_gb300 import shards, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ds = synth.workload("pan4x250")
    idx = oracle.IndexB(ds, oracle.choose_k(ds.n_residues), n_threads=2)
    mine = np.arange(rank, ds.n_genes, world, dtype=np.uint32)
    qrp, qcols, qs = oracle.best_hits_b(idx, mine)
    # the piece: a CSR over every gene, empty rows for the other ranks' genes
    lens = np.zeros(ds.n_genes, np.int64)
    lens[mine] = np.diff(qrp)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pieces = shards.gather_pieces(rp, qcols, qs)
    if rank == 0:
        out = {}
        for r, (prp, pc, pv) in enumerate(pieces):
            out[f"rp{r}"], out[f"c{r}"], out[f"s{r}"] = prp.numpy(), pc.numpy(), pv.numpy()
        np.savez(os.path.join(out_dir, "pieces.npz"), **out)
    else:
        assert pieces is None
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_one_dataset(tmp_path):
    """The union of the two ranks' gathered pieces is the single-process
    result: every row (columns and sum-min) and, from the merged rows, every
    BBH pair."""
    world = 2
    mp.spawn(_shard_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import oracle
    from paper_2510_23679_gb300 import synth
    ds = synth.workload("pan4x250")
    want_rp, want_c, want_s, want_bbh = oracle.all_pairs_b(oracle.IndexB(ds, oracle.choose_k(ds.n_residues)))
    z = np.load(tmp_path / "pieces.npz")
    G = ds.n_genes
    rows = {}
    for r in range(world):
        rp, c, s = z[f"rp{r}"], z[f"c{r}"], z[f"s{r}"]
        assert rp.shape == (G + 1,) and rp[-1] == len(c) == len(s)
        for g in np.flatnonzero(np.diff(rp)):
            assert g % world == r and g not in rows  # each row from its own rank only
            rows[int(g)] = (c[rp[g]:rp[g + 1]].tolist(), s[rp[g]:rp[g + 1]].astype(np.uint32).tolist())
    for g in range(G):
        assert rows.get(g, ([], [])) == (want_c[want_rp[g]:want_rp[g + 1]].tolist(),
                                         want_s[want_rp[g]:want_rp[g + 1]].tolist()), g
    gp = ds.genome_ptr
    genome = np.searchsorted(gp, np.arange(G), side="right") - 1
    bbh = sorted((a, b) for a, (cs, _) in rows.items() for b in cs
                 if genome[b] > genome[a] and a in rows.get(b, ([], []))[0])
    assert bbh == [tuple(p) for p in want_bbh.tolist()]
