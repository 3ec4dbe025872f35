"""Failure paths of the library, made on the host (no GPU fault is involved).

* Device memory: the context's allocator hook refuses the n-th allocation.
  The call that asked for it must fail with PD_ERR_OOM, release every
  temporary it had taken, and leave the context usable: the same context
  then produces exactly the result of an undisturbed context.
* Device errors recorded by kernels are covered by test_gpu_parity
  (bad letters, genes too long, malformed offsets); a bounded wait that
  expires (PD_ERR_TIMEOUT) by test_gpu_serve.
"""
import numpy as np
import pytest

from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


class Refuser:
    """Counts the library's allocations; refuses the `fail_at`-th (1-based)."""

    def __init__(self):
        self.fail_at = 0
        self.calls = 0
        self.granted = 0
        self.freed = 0

    def on_alloc(self, nbytes):
        self.calls += 1
        if self.calls == self.fail_at:
            return False
        self.granted += 1
        return True

    def on_free(self, ptr):
        self.freed += 1

    @property
    def live(self):
        return self.granted - self.freed


def _path(ctx, ds, k):
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    hits = pd.pd_best_hits_all(ctx, prof)
    rp, cols, s = pd.pd_hits_copy(ctx, hits)
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits))
    return rp, cols, s, bbh


def _attempt(ctx, ds, k):
    """Status of one whole pass.  The exception (and with it the traceback
    that would keep the pass's handles alive) ends inside this function."""
    try:
        _path(ctx, ds, k)
        return 0
    except pd.PdError as err:
        return err.status


def test_oom_from_the_allocator_hook_leaves_the_context_usable():
    import gc
    ds = synth.workload("pan4x250")
    k = 5
    want = _path(pd.pd_ctx_create(0), ds, k)
    ref = Refuser()
    ctx = pd.pd_ctx_create(0, on_alloc=ref.on_alloc, on_free=ref.on_free)
    _path(ctx, ds, k)
    gc.collect()
    n_allocs = ref.calls  # allocations of one whole pass
    assert n_allocs > 10 and ref.live == 0
    failed = 0
    for fail_at in sorted({1, 2, 3, n_allocs // 3, n_allocs // 2, n_allocs - 1, n_allocs}):
        ref.calls, ref.granted, ref.freed, ref.fail_at = 0, 0, 0, fail_at
        status = _attempt(ctx, ds, k)
        assert status == 5, f"refused allocation {fail_at}: status {status}"  # PD_ERR_OOM
        failed += 1
        gc.collect()
        assert ref.live == 0, f"refused allocation {fail_at}: {ref.live} allocations not released"
        ref.fail_at = 0
        got = _path(ctx, ds, k)
        for a, b in zip(got, want):
            assert np.array_equal(a, b), f"context unusable after refused allocation {fail_at}"
        gc.collect()
    assert failed >= 5


def test_oom_in_the_noalloc_set_up_is_impossible():
    """The allocation-free call takes nothing from the hook, so a hook that
    refuses everything does not affect it."""
    import torch
    ds = synth.workload("pan4x250")
    ref = Refuser()
    ctx = pd.pd_ctx_create(0, on_alloc=ref.on_alloc, on_free=ref.on_free)
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    want_rp, want_cols, want_s = pd.pd_hits_copy(ctx, pd.pd_best_hits(ctx, prof, 0, 1))
    ref.fail_at = ref.calls + 1  # the next allocation would be refused
    n_rows = int(ds.genome_ptr[1] - ds.genome_ptr[0])
    row_ptr = torch.zeros(n_rows + 1, dtype=torch.int64, device="cuda")
    cols = torch.zeros(4096, dtype=torch.int32, device="cuda")
    s = torch.zeros(4096, dtype=torch.int32, device="cuda")
    calls0 = ref.calls
    n = pd.pd_best_hits_noalloc(ctx, prof, 0, 1, row_ptr, cols, s)
    assert ref.calls == calls0
    assert n == len(want_cols)
    assert np.array_equal(row_ptr.cpu().numpy(), want_rp)
    assert np.array_equal(cols[:n].cpu().numpy(), want_cols)
