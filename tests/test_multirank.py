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
