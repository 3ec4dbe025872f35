"""The symmetric all-pairs form of pd_best_hits_all (each unordered genome
pair walked from one side; reverse Best Hits from the kept column maxima and
their exact ties) gives exactly the rows and BBH pairs of the form that walks
every genome from every query -- which the parity tests pin to the oracle --
on datasets rich in exact ties, empty genomes and tie lists larger than the
first allocation.  The whole-workload parity tests run the symmetric form
(the default) against oracle B as well."""
import numpy as np
import pytest

from paper_2510_23679_gb300 import pd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    sym = pd.pd_ctx_create(0)
    full = pd.pd_ctx_create(0)
    pd.pd_ctx_set_symmetric(full, False)
    return sym, full


def _run(ctx, ds, k):
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    hits = pd.pd_best_hits_all(ctx, prof)
    rp, cols, s = pd.pd_hits_copy(ctx, hits)
    bbh = pd.pd_bbh_copy(ctx, pd.pd_bbh_all(ctx, prof, hits))
    return rp, cols, s, bbh, pd.pd_hits_get_info(hits)


def _same(ctxs, ds, k):
    a = _run(ctxs[0], ds, k)
    b = _run(ctxs[1], ds, k)
    for x, y, name in zip(a[:4], b[:4], ("row_ptr", "cols", "s", "bbh")):
        assert np.array_equal(x, y), name
    return a, b


def test_pan4x250(ctxs):
    ds = synth.workload("pan4x250")
    a, b = _same(ctxs, ds, 5)
    # the symmetric form walks each unordered pair once (and never the own genome)
    assert a[4].postings_walked < 0.6 * b[4].postings_walked


@pytest.mark.parametrize("seed", range(8))
def test_random_tiny_with_ties(ctxs, seed):
    ds = synth.random_tiny(100 + seed, n_genomes=3 + seed % 3, max_genes=9, max_len=24,
                           letters=b"ACD" if seed % 2 else b"ACDE")
    for k in (1, 2, 3):
        _same(ctxs, ds, k)


def test_identical_genes_and_empty_genomes(ctxs):
    x, y = b"ACDEFGHIKL", b"MNPQRSTVWY"
    ds = synth.from_strings([[x, x, y], [], [x] * 5 + [y], [y, b"AC"], [], [x, x, x]])
    _same(ctxs, ds, 3)


def test_tie_list_larger_than_its_first_allocation(ctxs):
    """Every gene of genome 1 ties with all 300 genes of genome 0: about 90k
    ties, more than the first tie list holds (65536); the launch reruns."""
    ds = synth.from_strings([[b"ACDEFGHIK"] * 300, [b"ACDEFGHIK"] * 300])
    a, _ = _same(ctxs, ds, 4)
    assert len(a[1]) == 2 * 300 * 300  # every gene ties with every gene of the other genome


@pytest.mark.parametrize("symmetric", [True, False])
def test_walk_modes_same_bytes(symmetric):
    """Both posting walks of the sum-min kernel (forced through
    pd_ctx_set_walk), in both all-pairs forms, give the automatic choice's
    bytes -- on a dataset whose lists are long enough that the automatic
    choice is the warp walk for some queries and short enough that lists of
    one or two postings are common."""
    ds = synth.workload("pan4x250", seed=11)
    k = 4
    runs = []
    for mode in (pd.PD_WALK_AUTO, pd.PD_WALK_MERGE, pd.PD_WALK_WARP):
        ctx = pd.pd_ctx_create(0)
        pd.pd_ctx_set_symmetric(ctx, symmetric)
        pd.pd_ctx_set_walk(ctx, mode)
        runs.append(_run(ctx, ds, k))
    for r in runs[1:]:
        for x, y, name in zip(runs[0][:4], r[:4], ("row_ptr", "cols", "s", "bbh")):
            assert np.array_equal(x, y), name
    with pytest.raises(pd.PdError):
        pd.pd_ctx_set_walk(pd.pd_ctx_create(0), 3)
