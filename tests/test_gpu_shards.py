"""One dataset's all-against-all Best Hits split by query genes
(pd_best_hits_shard), reassembled (pd_hits_import) and finished with BBH
(pd_bbh_all): the result equals the unsplit run bit for bit, whether the
shards run in one process or in two processes (gloo ranks) sharing the GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ds = synth.workload("pan4x250")
    ctx = pd.pd_ctx_create(0)
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    hits = pd.pd_best_hits_all(ctx, prof)
    want = pd.pd_hits_copy(ctx, hits)
    want_bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits))
    return ds, ctx, prof, want, want_bbh


@pytest.mark.parametrize("n_shards", [1, 2, 3, 7])
def test_shards_reassemble_to_the_whole(setup, n_shards):
    ds, ctx, prof, (wrp, wcols, ws), want_bbh = setup
    pieces = [pd.pd_hits_copy(ctx, pd.pd_best_hits_shard(ctx, prof, r, n_shards)) for r in range(n_shards)]
    owner = np.full(ds.n_genes, -1)
    for r, (rp, cols, s) in enumerate(pieces):
        nonempty = np.flatnonzero(np.diff(rp))
        assert np.all(owner[nonempty] == -1), "a row in two shards"
        owner[nonempty] = r
    assert np.array_equal(owner >= 0, np.diff(wrp) > 0)
    merged = pd.pd_hits_import(ctx, prof, pieces)
    rp, cols, s = pd.pd_hits_copy(ctx, merged)
    assert np.array_equal(rp, wrp) and np.array_equal(cols, wcols) and np.array_equal(s, ws)
    assert np.array_equal(pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, merged)), want_bbh)


def test_import_rejects_malformed_pieces(setup):
    ds, ctx, prof, (wrp, wcols, ws), _ = setup
    with pytest.raises(pd.PdError) as e:  # every row twice
        pd.pd_hits_import(ctx, prof, [(wrp, wcols, ws), (wrp, wcols, ws)])
    assert e.value.status == 1
    row = int(np.flatnonzero(np.diff(wrp) >= 2)[0])
    bad = wcols.copy()
    bad[wrp[row]], bad[wrp[row] + 1] = bad[wrp[row] + 1], bad[wrp[row]]
    with pytest.raises(pd.PdError) as e:  # a row not ascending
        pd.pd_hits_import(ctx, prof, [(wrp, bad, ws)])
    assert e.value.status == 1
    bad = wcols.copy()
    bad[0] = ds.n_genes
    with pytest.raises(pd.PdError) as e:  # a column outside the dataset
        pd.pd_hits_import(ctx, prof, [(wrp, bad, ws)])
    assert e.value.status == 1
    with pytest.raises(pd.PdError) as e:
        pd.pd_best_hits_shard(ctx, prof, 3, 3)
    assert e.value.status == 1
    # the context stays usable
    again = pd.pd_hits_copy(ctx, pd.pd_hits_import(ctx, prof, [(wrp, wcols, ws)]))
    assert np.array_equal(again[1], wcols)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2510_23679_gb300 import shards
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)  # both ranks on the one GPU: their kernels never wait on each other
    ds = synth.workload("pan4x250")
    ctx = pd.pd_ctx_create(0)
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    hits, bbh = shards.sharded_bbh(ctx, prof)
    if rank == 0:
        rp, cols, s = pd.pd_hits_copy(ctx, hits)
        np.savez(os.path.join(out_dir, "sharded.npz"), rp=rp, cols=cols, s=s, bbh=pd.pd_bbh_copy(ctx, bbh))
    else:
        assert hits is None and bbh is None
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu(setup, tmp_path):
    _, _, _, (wrp, wcols, ws), want_bbh = setup
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    z = np.load(tmp_path / "sharded.npz")
    assert np.array_equal(z["rp"], wrp) and np.array_equal(z["cols"], wcols) and np.array_equal(z["s"], ws)
    assert np.array_equal(z["bbh"], want_bbh)
