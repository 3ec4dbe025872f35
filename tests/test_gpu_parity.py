"""GPU path (through the C ABI) against the CPU oracle: bit-exact.

Every sum-min, every Best Hit index and every Bidirectional Best Hit pair must
equal the oracle's; the multiplicity vectors and the inverted index must equal
the oracle's k-mer counts.  Sizes span several thread-block tiles with ragged
tails (genes of 80..600 residues, 250 genes per genome) plus the edge cases:
k = 1, genes shorter than k, empty genes, ties, rows without candidates,
inputs that overflow the shared-memory accumulator, saturated posting counts.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2510_23679_gb300 import pd, synth
from tests import _golden
from tests._gpu import DeviceRun, all_pairs_row_slice, csr_lists, oracle_nonzero, oracle_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = pd.pd_ctx_create(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pan4(ctx):
    ds = synth.workload("pan4x250")
    k = oracle.choose_k(ds.n_residues)
    assert k == 5
    run = DeviceRun(ctx, ds, k)
    pairs = list(itertools.permutations(range(ds.n_genomes), 2))
    return run, oracle_pairs(ds, k, pairs, n_threads=4)


# ------------------------------------------------------------------ hand-worked examples
@pytest.mark.parametrize("fname", _golden.all_fixtures())
def test_golden_on_gpu(ctx, fname):
    g = _golden.load(fname)
    ds = synth.from_strings([g.rows, g.cols])
    run = DeviceRun(ctx, ds, g.k)
    want = {(a, b): s for a, row in enumerate(g.S) for b, (s, _) in enumerate(row) if s > 0}
    assert run.summin(0, 1) == want
    rows, _ = run.best_hits(0, 1)
    assert rows == g.row_bh
    cols, _ = run.best_hits(1, 0)
    assert cols == g.col_bh
    assert run.bbh(0, 1) == g.bbh
    rp, cbh, s, bbh, _ = run.all_pairs()
    nr = len(g.rows)
    assert [all_pairs_row_slice(ds, rp, cbh, a, 1) for a in range(nr)] == g.row_bh
    assert [tuple(x) for x in bbh.tolist()] == [(a, nr + b) for a, b in g.bbh]


# ------------------------------------------------------------------ profiles
def test_multiplicity_vectors(pan4, ctx):
    run, _ = pan4
    ds = run.ds
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, run.k)
    mv, La = run.mv()
    for g in range(ds.n_genes):
        kmers, cnt = prof.mv(g)
        assert mv[g][0] == kmers and mv[g][1] == cnt.tolist(), f"gene {g}"
        assert La[g] == prof.La(g)
    assert run.info.n_windows == sum(prof.La(g) for g in range(ds.n_genes))


def test_inverted_index(pan4, ctx):
    run, _ = pan4
    ds = run.ds
    prof = oracle.Profiles(ds.residues, ds.gene_ptr, run.k)
    expect = {}
    for g in range(ds.n_genes):
        kmers, cnt = prof.mv(g)
        for km, c in zip(kmers, cnt):
            expect.setdefault(km, []).append((g, int(c)))
    post_ptr, codes, genes, counts = pd.pd_profiles_copy_index(ctx, run.prof)
    got = {}
    from tests._gpu import decode_code
    for w in range(len(codes)):
        km = decode_code(int(codes[w]), run.k)
        got[km] = list(zip(genes[post_ptr[w]:post_ptr[w + 1]].tolist(), counts[post_ptr[w]:post_ptr[w + 1]].tolist()))
    assert got == expect
    assert list(codes) == sorted(codes)
    assert run.info.n_distinct == len(expect)


# ------------------------------------------------------------------ sum-min, BH, BBH per genome pair
def test_summin_every_pair(pan4):
    run, ref = pan4
    for (gi, gj), R in ref.items():
        assert run.summin(gi, gj) == oracle_nonzero(R), f"pair {gi},{gj}"


def test_best_hits_every_pair(pan4):
    run, ref = pan4
    for (gi, gj), R in ref.items():
        rows, svals = run.best_hits(gi, gj)
        assert rows == csr_lists(R.row_ptr, R.row_col), f"pair {gi},{gj}"
        for a, (cols, ss) in enumerate(zip(rows, svals)):
            assert ss == [int(R.S[a, b]) for b in cols]


def test_bbh_every_pair(pan4):
    run, ref = pan4
    for (gi, gj), R in ref.items():
        assert run.bbh(gi, gj) == [tuple(x) for x in R.bbh.tolist()], f"pair {gi},{gj}"


def test_all_pairs_equals_oracle(pan4):
    run, ref = pan4
    ds = run.ds
    rp, cols, s, bbh, info = run.all_pairs()
    gp = ds.genome_ptr
    for (gi, gj), R in ref.items():
        got = [all_pairs_row_slice(ds, rp, cols, int(gp[gi]) + a, gj) for a in range(R.S.shape[0])]
        assert got == csr_lists(R.row_ptr, R.row_col), f"pair {gi},{gj}"
    want = []
    for gi, gj in itertools.combinations(range(ds.n_genomes), 2):
        want += [(int(gp[gi]) + a, int(gp[gj]) + b) for a, b in ref[(gi, gj)].bbh.tolist()]
    assert [tuple(x) for x in bbh.tolist()] == sorted(want)
    assert info.n_deferred == 0


def test_all_pairs_is_deterministic(pan4):
    run, _ = pan4
    r1 = run.all_pairs()
    r2 = run.all_pairs()
    for x, y in zip(r1[:4], r2[:4]):
        assert np.array_equal(x, y)


def test_device_inputs_match_host_inputs(pan4, ctx):
    run, _ = pan4
    dev = DeviceRun(ctx, run.ds, run.k, device_inputs=True)
    for x, y in zip(run.all_pairs()[:4], dev.all_pairs()[:4]):
        assert np.array_equal(x, y)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_tiny_random_against_oracle(ctx, seed, k):
    letters = [b"AC", b"ACD", b"ACDEFGHIKL", synth.ALPHABET][seed % 4]
    ds = synth.random_tiny(1000 + seed * 3 + k, n_genomes=3, max_genes=7, max_len=40, letters=letters)
    run = DeviceRun(ctx, ds, k)
    pairs = list(itertools.permutations(range(ds.n_genomes), 2))
    ref = oracle_pairs(ds, k, pairs)
    for (gi, gj), R in ref.items():
        assert run.summin(gi, gj) == oracle_nonzero(R)
        assert run.best_hits(gi, gj)[0] == csr_lists(R.row_ptr, R.row_col)
        assert run.bbh(gi, gj) == [tuple(x) for x in R.bbh.tolist()]
    rp, cols, s, bbh, _ = run.all_pairs()
    gp = ds.genome_ptr
    for (gi, gj), R in ref.items():
        got = [all_pairs_row_slice(ds, rp, cols, int(gp[gi]) + a, gj) for a in range(R.S.shape[0])]
        assert got == csr_lists(R.row_ptr, R.row_col)


def test_empty_genes_and_genomes(ctx):
    ds = synth.from_strings([[b"", b"ACDEF", b"A"], [], [b"ACDEG", b""], [b"CDEF"]])
    run = DeviceRun(ctx, ds, 3)
    ref = oracle_pairs(ds, 3, [(0, 2), (2, 0), (0, 3), (2, 3)])
    for (gi, gj), R in ref.items():
        assert run.summin(gi, gj) == oracle_nonzero(R)
        assert run.bbh(gi, gj) == [tuple(x) for x in R.bbh.tolist()]
    rp, cols, s, bbh, _ = run.all_pairs()
    assert len(rp) == ds.n_genes + 1
    assert run.best_hits(0, 1)[0] == [[], [], []]  # empty target genome


def test_k_equal_to_gene_length(ctx):
    ds = synth.from_strings([[b"ACDEFGHIKL", b"ACDEFGHIKM"], [b"ACDEFGHIKL", b"ACDEFGHIK"]])
    run = DeviceRun(ctx, ds, 8)
    ref = oracle_pairs(ds, 8, [(0, 1)])[(0, 1)]
    assert run.summin(0, 1) == oracle_nonzero(ref)
    assert run.bbh(0, 1) == [tuple(x) for x in ref.bbh.tolist()]


def test_errors_are_reported(ctx):
    bad = synth.from_strings([[b"ACDX"], [b"ACD"]])
    with pytest.raises(pd.PdError) as e:
        pd.pd_build_profiles(ctx, bad.residues, bad.gene_ptr, bad.genome_ptr, 2)
    assert e.value.status == 2
    ok = synth.from_strings([[b"ACD"], [b"ACD"]])
    for k in (0, pd.PD_MAX_K + 1):
        with pytest.raises(pd.PdError) as e:
            pd.pd_build_profiles(ctx, ok.residues, ok.gene_ptr, ok.genome_ptr, k)
        assert e.value.status == 4
    long = synth.from_strings([[b"A" * (pd.PD_MAX_WINDOWS + 2)], [b"A"]])
    with pytest.raises(pd.PdError) as e:
        pd.pd_build_profiles(ctx, long.residues, long.gene_ptr, long.genome_ptr, 1)
    assert e.value.status == 3
    run = DeviceRun(ctx, ok, 2)
    with pytest.raises(pd.PdError) as e:
        pd.pd_best_hits(ctx, run.prof, 0, 0)
    assert e.value.status == 1
    # the context stays usable after errors
    assert run.bbh(0, 1) == [(0, 0)]


def test_accumulator_overflow_takes_the_large_path(ctx):
    # one query shares a k-mer with 5000 distinct targets (> 3/4 of the shared
    # table) and ties with all of them (> the shared Best Hit list)
    rng = np.random.default_rng(7)
    letters = np.frombuffer(b"FGHIKLMNPQRSTVWY", np.uint8)
    targets = [b"AC" + rng.choice(letters, size=6).tobytes() for _ in range(5000)]
    ds = synth.from_strings([[b"ACDE", b"GGGG"], targets])
    run = DeviceRun(ctx, ds, 2)
    R = oracle_pairs(ds, 2, [(0, 1)])[(0, 1)]
    assert run.summin(0, 1) == oracle_nonzero(R)
    rows, _ = run.best_hits(0, 1)
    assert rows == csr_lists(R.row_ptr, R.row_col)
    assert run.bbh(0, 1) == [tuple(x) for x in R.bbh.tolist()]
    rp, cols, s, bbh, info = run.all_pairs()
    assert info.n_deferred >= 1
    assert [all_pairs_row_slice(ds, rp, cols, a, 1) for a in range(2)] == csr_lists(R.row_ptr, R.row_col)


def test_saturated_posting_counts_and_long_genes(ctx):
    # > 2^17 genes leave 14 count bits in a packed posting (cap 16383); two
    # long one-letter genes exceed it, so the exact count is looked up.
    n_empty = 70000
    ds = synth.from_strings([[b"A" * 20000] + [b""] * n_empty, [b"A" * 17000 + b"C"] + [b""] * n_empty])
    run = DeviceRun(ctx, ds, 1)
    assert run.info.count_bits == 14
    pair = synth.from_strings([[b"A" * 20000], [b"A" * 17000 + b"C"]])
    prof = oracle.Profiles(pair.residues, pair.gene_ptr, 1)
    s, d = prof.summin(0, 1)
    assert (s, d) == (17000, 20001)
    assert run.summin(0, 1) == {(0, 0): s}
    assert run.bbh(0, 1) == [(0, 0)]
    _, _, gen, cnt = pd.pd_profiles_copy_index(ctx, run.prof)
    assert sorted(cnt.tolist()) == [1, 17000, 20000]


@pytest.mark.parametrize("letter", "AHMRWY")
def test_saturated_count_in_a_gene_with_many_kmers(ctx, letter):
    """The exact count behind a saturated posting is looked up in the target
    gene's multiplicity vector, which is stored in hash order: a target with
    many distinct k-mers besides the saturated one must still be found, for
    small, middle and large k-mer ids."""
    n_empty = 70000
    sat = letter.encode()
    other = b"W" if sat != b"W" else b"A"
    tail = bytes(c for c in b"ACDEFGHIKLMNPQRSTVWY" if c != sat[0])
    target = sat * 20000 + tail * 3
    query = sat * 17000 + other
    ds = synth.from_strings([[query] + [b""] * n_empty, [target] + [b""] * n_empty])
    run = DeviceRun(ctx, ds, 1)
    assert run.info.count_bits == 14
    pair = synth.from_strings([[query], [target]])
    prof = oracle.Profiles(pair.residues, pair.gene_ptr, 1)
    s, _ = prof.summin(0, 1)
    assert s == 17001
    assert run.summin(0, 1) == {(0, 0): s}
    assert run.summin(1, 0) == {(0, 0): s}
    assert run.bbh(0, 1) == [(0, 0)]


@pytest.mark.parametrize("n_genes", [40, 3000, 20000])
def test_index_lists_of_every_length(ctx, n_genes):
    """Posting lists from 1 to n_genes entries (short lists, block-sorted lists
    and, past 8192 entries, lists sorted in global memory) come out in gene
    order with the right counts."""
    rng = np.random.default_rng(n_genes)
    letters = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", np.uint8)
    genes = []
    for g in range(n_genes):
        tail = letters[rng.integers(0, 20, size=int(rng.integers(0, 12)))].tobytes()
        genes.append(b"ACDEF" * int(1 + g % 3) + tail)  # every gene holds ACD, CDE, DEF
    ds = synth.from_strings([genes[: n_genes // 2], genes[n_genes // 2:]])
    k = 3
    prof = pd.pd_build_profiles(ctx, ds.residues, ds.gene_ptr, ds.genome_ptr, k)
    post_ptr, codes, g_out, c_out = pd.pd_profiles_copy_index(ctx, prof)
    ref = oracle.Profiles(ds.residues, ds.gene_ptr, k)
    expect = {}
    for g in range(ds.n_genes):
        kmers, cnt = ref.mv(g)
        for km, c in zip(kmers, cnt):
            expect.setdefault(km, []).append((g, int(c)))
    from tests._gpu import decode_code
    got = {decode_code(int(codes[w]), k): list(zip(g_out[post_ptr[w]:post_ptr[w + 1]].tolist(),
                                                   c_out[post_ptr[w]:post_ptr[w + 1]].tolist()))
           for w in range(len(codes))}
    assert got == expect
    assert max(len(v) for v in expect.values()) == n_genes


def test_malformed_offsets_are_errors(ctx):
    """Offsets are checked on the device before any kernel reads past them:
    decreasing, not starting at 0, not ending at n_res -- on host and device
    inputs -- and a genome_ptr that does not cover the genes."""
    import torch
    res = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY" * 5, np.uint8).copy()
    good_gp = np.array([0, 30, 60, 100], np.int64)
    gn = np.array([0, 2, 3], np.int32)
    bad_gps = [np.array([0, 30, 20, 100], np.int64), np.array([5, 30, 60, 100], np.int64),
               np.array([0, 30, 60, 99], np.int64), np.array([0, 30, 60, 10_000], np.int64)]
    for gp in bad_gps:
        for dev in (False, True):
            g = torch.from_numpy(gp).cuda() if dev else gp
            r = torch.from_numpy(res).cuda() if dev else res
            with pytest.raises(pd.PdError) as e:
                pd.pd_build_profiles(ctx, r, g, gn, 3)
            assert e.value.status == 1, (gp.tolist(), dev)
    for bad_gn in (np.array([0, 4, 3], np.int32), np.array([0, 2, 4], np.int32), np.array([1, 2, 3], np.int32)):
        for dev in (False, True):
            n = torch.from_numpy(bad_gn).cuda() if dev else bad_gn
            with pytest.raises(pd.PdError) as e:
                pd.pd_build_profiles(ctx, res, good_gp, n, 3)
            assert e.value.status == 1, (bad_gn.tolist(), dev)
    # the context stays usable
    prof = pd.pd_build_profiles(ctx, res, good_gp, gn, 3)
    assert pd.pd_profiles_get_info(prof).n_genes == 3


def test_kernel_timing_and_its_filter(pan4, ctx):
    """Per-launch timing: every kernel by default, or the launches of one
    kernel name; the filter changes no result."""
    run, _ = pan4
    prof = run.prof
    ref = pd.pd_hits_copy(ctx, pd.pd_best_hits_all(ctx, prof))
    pd.pd_ctx_reset_timing(ctx)
    pd.pd_ctx_set_timing(ctx, True)
    try:
        pd.pd_best_hits_all(ctx, prof)
        _, n_all = pd.pd_ctx_kernel_time(ctx, None)
        ms_bh, n_bh = pd.pd_ctx_kernel_time(ctx, "summin_bh")
        assert n_bh == 1 and ms_bh > 0 and n_all >= 2  # tier 1 and tier 2 at least
        pd.pd_ctx_reset_timing(ctx)
        pd.pd_ctx_set_timing_filter(ctx, "summin_bh")
        got = pd.pd_hits_copy(ctx, pd.pd_best_hits_all(ctx, prof))
        _, n_all = pd.pd_ctx_kernel_time(ctx, None)
        _, n_bh = pd.pd_ctx_kernel_time(ctx, "summin_bh")
        assert n_all == n_bh == 1
        assert all(np.array_equal(a, b) for a, b in zip(got, ref))
    finally:
        pd.pd_ctx_set_timing(ctx, False)
        pd.pd_ctx_set_timing_filter(ctx, None)
        pd.pd_ctx_reset_timing(ctx)


@pytest.mark.parametrize("better_first", [True, False])
def test_ratios_closer_than_float_resolution(ctx, better_first):
    """Eq. (8) compares ratios exactly.  Two targets at 60000/60001 and
    59999/60000 differ by 2.8e-10, less than a float's resolution there:
    only the larger is a Best Hit, in either gene order (k = 1, so s is the
    letter-count overlap)."""
    assert np.float32(60000) / np.float32(60001) == np.float32(59999) / np.float32(60000)
    rng = np.random.default_rng(7)
    letters = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", np.uint8)
    a = rng.choice(letters, 60000)
    better = np.concatenate([a, letters[:1]])  # s = 60000, den = 60000 + 60001 - 60000
    worse = a[:-1]                             # s = 59999, den = 60000 + 59999 - 59999
    genes = [a] + ([better, worse] if better_first else [worse, better])
    res = np.concatenate(genes).astype(np.uint8)
    gp = np.cumsum([0] + [len(g) for g in genes]).astype(np.int64)
    gn = np.array([0, 1, 3], np.int32)
    prof = pd.pd_build_profiles(ctx, res, gp, gn, 1)
    want = 1 if better_first else 2
    rp, cols, s = pd.pd_hits_copy(ctx, pd.pd_best_hits_all(ctx, prof))
    assert cols[rp[0]:rp[1]].tolist() == [want] and s[rp[0]:rp[1]].tolist() == [60000]
    rp, cols, s = pd.pd_hits_copy(ctx, pd.pd_best_hits(ctx, prof, 0, 1))
    assert cols[rp[0]:rp[1]].tolist() == [want - 1] and s[rp[0]:rp[1]].tolist() == [60000]
    # the oracle agrees
    ds = synth.Pangenome(res, gp, gn, np.full(3, -1, np.int32))
    assert oracle.pair_for_dataset(ds, 0, 1, 1).row_bh(0).tolist() == [want - 1]


@pytest.mark.parametrize("n_targets,n_tied", [(3000, 440), (3100, 460), (1000, 447), (1000, 449)])
def test_occupied_list_and_hit_list_bounds(ctx, n_targets, n_tied):
    """A query sharing one k-mer with n_targets genes, n_tied of them at the
    shortest length (so tied Best Hits): around the tier-1 bounds of 3072
    listed slots and 448 hits, every count gives the oracle's answer."""
    rng = np.random.default_rng(n_targets + n_tied)
    letters = np.frombuffer(b"FGHIKLMNPQRSTVWY", np.uint8)
    targets = []
    for t in range(n_targets):
        extra = 6 if t < n_tied else 7 + int(rng.integers(0, 20))
        targets.append(b"AC" + rng.choice(letters, size=extra).tobytes())
    ds = synth.from_strings([[b"ACDE", b"GGGG"], targets])
    run = DeviceRun(ctx, ds, 2)
    R = oracle_pairs(ds, 2, [(0, 1)])[(0, 1)]
    rows, _ = run.best_hits(0, 1)
    assert rows == csr_lists(R.row_ptr, R.row_col)
    assert len(rows[0]) == n_tied
    rp, cols, s, bbh, info = run.all_pairs()
    assert [all_pairs_row_slice(ds, rp, cols, a, 1) for a in range(2)] == csr_lists(R.row_ptr, R.row_col)


@pytest.mark.parametrize("n_genomes", [80, 100])
def test_both_tier1_layouts_against_oracle(ctx, n_genomes):
    """Datasets below and above the genome count at which tier 1 switches from
    its compact to its full shared-memory layout: all-pairs Best Hits and BBH
    equal the oracle on sampled genome pairs."""
    ds = synth.generate(n_genomes=n_genomes, genes_per_genome=("fixed", 12), n_families=30,
                        length_dist=("uniform", 40, 160), core_frac=0.5, accessory_draw=None, subst_max=0.2,
                        indel_max=0.03, paralog_frac=0.1, singleton_frac=0.05, seed=11)
    k = 3
    run = DeviceRun(ctx, ds, k)
    rp, cols, s, bbh, info = run.all_pairs()
    for gi, gj in [(0, 1), (n_genomes - 1, 0), (37, n_genomes - 2)]:
        R = oracle.pair_for_dataset(ds, gi, gj, k)
        g0 = int(ds.genome_ptr[gi])
        rows = [all_pairs_row_slice(ds, rp, cols, g0 + a, gj) for a in range(R.S.shape[0])]
        assert rows == csr_lists(R.row_ptr, R.row_col), (gi, gj)
        assert run.bbh(gi, gj) == [tuple(x) for x in R.bbh.tolist()], (gi, gj)
