"""pd_best_hits_noalloc: the allocation-free form of pd_best_hits.

Some callers of this library cannot allocate device memory while they run
(their device memory belongs to an external pool, or an allocation in a
latency-critical loop could block or fail).  For them the library offers one
entry point whose temporaries live in a fixed scratch array and whose results
go to caller-owned buffers.  This file checks, through the C ABI, that it
returns exactly what pd_best_hits + pd_hits_copy return, on two calls in a
row, and that it rejects sizes beyond its limits.  It is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    ctx = pd.pd_ctx_create(0)
    ds = synth.workload("pan4x250")
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    return torch, ctx, ds, prof


@pytest.mark.parametrize("gi,gj", [(0, 1), (3, 2)])
def test_noalloc_equals_best_hits_twice(setup, gi, gj):
    torch, ctx, ds, prof = setup
    ref_ptr, ref_cols, ref_s = pd.pd_hits_copy(ctx, pd.pd_best_hits(ctx, prof, gi, gj))
    n_rows = int(ds.genome_ptr[gi + 1] - ds.genome_ptr[gi])
    for call in range(2):
        row_ptr = torch.full((n_rows + 1,), -1, dtype=torch.int64, device="cuda")
        cols = torch.full((4096,), -1, dtype=torch.int32, device="cuda")
        s = torch.full((4096,), -1, dtype=torch.int32, device="cuda")
        n = pd.pd_best_hits_noalloc(ctx, prof, gi, gj, row_ptr, cols, s)
        torch.cuda.synchronize()
        assert n == len(ref_cols), f"call {call}"
        assert np.array_equal(row_ptr.cpu().numpy(), ref_ptr), f"call {call}"
        assert np.array_equal(cols[:n].cpu().numpy(), ref_cols), f"call {call}"
        assert np.array_equal(s[:n].cpu().numpy().astype(np.uint32), ref_s), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_limits(setup):
    torch, ctx, _, _ = setup
    # a query genome with more genes than PD_NOALLOC_MAX_ROWS (empty genes are cheap)
    big = synth.from_strings([[b"ACDEFG"] + [b""] * pd.PD_NOALLOC_MAX_ROWS, [b"ACDEFG"]])
    prof = pd.pd_build_profiles(ctx, big.residues, big.gene_ptr, big.genome_ptr, 3)
    row_ptr = torch.zeros(pd.PD_NOALLOC_MAX_ROWS + 2, dtype=torch.int64, device="cuda")
    cols = torch.zeros(16, dtype=torch.int32, device="cuda")
    s = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(pd.PdError) as e:
        pd.pd_best_hits_noalloc(ctx, prof, 0, 1, row_ptr, cols, s)
    assert e.value.status == 1 and "PD_NOALLOC_MAX_ROWS" in str(e.value)
    # ... and a target genome beyond PD_NOALLOC_MAX_TARGETS
    with pytest.raises(pd.PdError) as e:
        pd.pd_best_hits_noalloc(ctx, prof, 1, 0, row_ptr[:2], cols, s)
    assert e.value.status == 1 and "PD_NOALLOC_MAX_TARGETS" in str(e.value)
    # an output smaller than the result is refused (every row ties with all 3 targets)
    small = synth.from_strings([[b"ACDEFGH", b"ACDEFGH"], [b"ACDEFGH", b"ACDEFGH", b"ACDEFGH"]])
    prof2 = pd.pd_build_profiles(ctx, small.residues, small.gene_ptr, small.genome_ptr, 2)
    with pytest.raises(pd.PdError) as e:
        pd.pd_best_hits_noalloc(ctx, prof2, 0, 1, row_ptr[:3], cols[:2], s[:2])
    assert e.value.status == 1
