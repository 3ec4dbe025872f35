"""Pins of the oracle's family extraction (connected components of the BBH
graph, labelled by their smallest gene id): hand-made graphs with known
components, and random graphs against scipy's connected-components routine."""
import numpy as np
import pytest

import oracle


def test_hand_made_graphs():
    assert oracle.families(4, []).tolist() == [0, 1, 2, 3]
    # a path 3-1-4 and a separate pair 0-2, plus an isolated node 5
    assert oracle.families(6, [(3, 1), (1, 4), (2, 0)]).tolist() == [0, 1, 0, 1, 1, 5]
    # duplicate edges, self-loops and a cycle
    assert oracle.families(5, [(4, 3), (3, 4), (2, 2), (3, 2), (2, 4)]).tolist() == [0, 1, 2, 2, 2]


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_against_scipy(seed):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 2 * n))
    a, b = rng.integers(0, n, size=m), rng.integers(0, n, size=m)
    lab = oracle.families(n, zip(a, b))
    g = coo_matrix((np.ones(m), (a, b)), shape=(n, n))
    nc, ref = connected_components(g, directed=False)
    assert len(np.unique(lab)) == nc
    # same partition, and each label is the smallest member of its part
    for c in range(nc):
        members = np.flatnonzero(ref == c)
        assert np.all(lab[members] == members.min())


def test_all_pairs_bbh_matches_pairs():
    from paper_2510_23679_gb300 import synth
    ds = synth.random_tiny(3, n_genomes=3, max_genes=5, max_len=30, letters=b"ACDE")
    k = 2
    pairs = oracle.all_pairs_bbh(ds, k)
    gp = ds.genome_ptr
    R = oracle.pair_for_dataset(ds, 0, 2, k)
    sel = (pairs[:, 0] < gp[1]) & (pairs[:, 1] >= gp[2])
    assert (pairs[sel] - [0, int(gp[2])]).tolist() == R.bbh.tolist()
