"""pd_best_hits_noalloc: the allocation-free form of pd_best_hits.

Some callers of this library cannot allocate device memory while they run
(their device memory belongs to an external pool, or an allocation in a
latency-critical loop could block or fail).  For them the library offers one
entry point whose temporaries live in a fixed scratch array and whose results
go to caller-owned buffers.  This file checks, through the C ABI, that it
returns exactly what pd_best_hits + pd_hits_copy return, on two calls in a
row; that neither call asks the context's allocator for memory (the context
is created with counting allocator hooks); that the global-memory tier carved
out of the scratch array gives the same result when queries reach it; that an
empty query genome gives an empty result; and that sizes beyond the limits are
refused.  It is collected last so a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


class AllocCounter:
    def __init__(self):
        self.allocs = 0
        self.frees = 0

    def on_alloc(self, nbytes):
        self.allocs += 1
        return True

    def on_free(self, ptr):
        self.frees += 1


@pytest.fixture(scope="module")
def setup():
    import torch
    counter = AllocCounter()
    ctx = pd.pd_ctx_create(0, on_alloc=counter.on_alloc, on_free=counter.on_free)
    ds = synth.workload("pan4x250")
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, 5)
    assert counter.allocs > 0  # the hooks do see the library's allocations
    return torch, ctx, ds, prof, counter


def _device_out(torch, n_rows, cap):
    return (torch.full((n_rows + 1,), -1, dtype=torch.int64, device="cuda"),
            torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
            torch.full((cap,), -1, dtype=torch.int32, device="cuda"))


def _check_equal(torch, ctx, prof, gi, gj, n_rows, cap, counter, calls=2):
    ref_ptr, ref_cols, ref_s = pd.pd_hits_copy(ctx, pd.pd_best_hits(ctx, prof, gi, gj))
    outs = [_device_out(torch, n_rows, cap) for _ in range(calls)]  # allocated by torch, before the calls
    torch.cuda.synchronize()
    launches = []
    for call, (row_ptr, cols, s) in enumerate(outs):
        before = (counter.allocs, counter.frees)
        l0 = pd.pd_ctx_launch_count(ctx)
        n = pd.pd_best_hits_noalloc(ctx, prof, gi, gj, row_ptr, cols, s)
        launches.append(pd.pd_ctx_launch_count(ctx) - l0)
        assert (counter.allocs, counter.frees) == before, f"call {call} used the context's allocator"
        torch.cuda.synchronize()
        assert n == len(ref_cols), f"call {call}"
        assert np.array_equal(row_ptr.cpu().numpy(), ref_ptr), f"call {call}"
        assert np.array_equal(cols[:n].cpu().numpy(), ref_cols), f"call {call}"
        assert np.array_equal(s[:n].cpu().numpy().astype(np.uint32), ref_s), f"call {call}"
    return launches


@pytest.mark.parametrize("gi,gj", [(0, 1), (3, 2)])
def test_noalloc_equals_best_hits_twice_without_allocating(setup, gi, gj):
    torch, ctx, ds, prof, counter = setup
    n_rows = int(ds.genome_ptr[gi + 1] - ds.genome_ptr[gi])
    _check_equal(torch, ctx, prof, gi, gj, n_rows, 4096, counter)


def test_noalloc_global_tier_in_the_scratch_array(setup):
    """Queries the shared-memory tiers defer reach the global-memory tier,
    whose tables live in the scratch array: (a) 5000 tied Best Hits per query
    (more than tier 2's hit list), (b) 20000 distinct targets per query (more
    than tier 2's 16384-slot table).  Each has a twin with the same number of
    query genes and some Best Hits that stays in shared memory: the deferred
    calls launch exactly one kernel more (the global tier)."""
    torch, ctx, _, _, counter = setup
    rng = np.random.default_rng(3)
    filler = np.frombuffer(b"KLMNPQRSTVWY", np.uint8)

    def rand_gene(n):
        return filler[rng.integers(0, filler.size, size=n)].tobytes()

    cases = {
        # query genes tie with all 5000 identical targets / with none of 5000 distinct ones
        "ties": ([[b"ACDEFGH"] * 3, [b"ACDEFGH"] * 5000],
                 [[b"ACDEFGH"] * 3, [b"ACDEFGH"] + [rand_gene(7) for _ in range(4999)]]),
        # every target shares exactly the k-mer ACD with the query genes (s = 1), lengths 4..13
        "wide": ([[b"ACDE", b"ACDEY"], [b"ACD" + rand_gene(int(rng.integers(1, 11))) for _ in range(20000)]],
                 [[b"ACDE", b"ACDEY"], [b"ACD" + rand_gene(int(rng.integers(1, 11))) for _ in range(10)]]),
    }
    for name, (deferred, plain) in cases.items():
        per_case = []
        for genomes in (deferred, plain):
            d = synth.from_strings(genomes)
            prof = pd.pd_build_profiles(ctx, d.residues, d.gene_ptr, d.genome_ptr, 3)
            per_case.append(_check_equal(torch, ctx, prof, 0, 1, len(genomes[0]), 1 << 16, counter))
        assert per_case[0][0] == per_case[1][0] + 1, f"{name}: the global tier did not run ({per_case})"
        assert per_case[0][1] == per_case[0][0], name


def test_noalloc_empty_query_genome(setup):
    torch, ctx, _, _, counter = setup
    for genomes in ([[], [b"ACDEFGH", b"KLMN"]], [[b"AC", b"D", b""], [b"ACDEFGH"]]):
        d = synth.from_strings(genomes)
        prof = pd.pd_build_profiles(ctx, d.residues, d.gene_ptr, d.genome_ptr, 3)
        n_rows = len(genomes[0])
        row_ptr, cols, s = _device_out(torch, n_rows, 16)
        before = counter.allocs
        n = pd.pd_best_hits_noalloc(ctx, prof, 0, 1, row_ptr, cols, s)
        torch.cuda.synchronize()
        assert counter.allocs == before
        assert n == 0
        assert row_ptr.cpu().numpy().tolist() == [0] * (n_rows + 1)


def test_noalloc_rejects_sizes_beyond_its_limits(setup):
    torch, ctx, _, _, _ = setup
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
    # buffers the binding refuses before the call: host memory, a short row_ptr
    with pytest.raises(ValueError):
        pd.pd_best_hits_noalloc(ctx, prof2, 0, 1, torch.zeros(3, dtype=torch.int64), cols, s)
    with pytest.raises(ValueError):
        pd.pd_best_hits_noalloc(ctx, prof2, 0, 1, row_ptr[:2], cols, s)
