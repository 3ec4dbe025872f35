"""Pins of the oracle's candidate filters: the length threshold theta of
Eq. (6) and the directional threshold tau of Eq. (7), against a hand-worked
case and against brute force (windows listed one by one, exact fractions)."""
from fractions import Fraction

import pytest

import oracle
from paper_2510_23679_gb300 import synth
from tests.test_oracle_pins import brute_summax, brute_summin, windows


def brute_p(s: bytes, t: bytes, k: int) -> Fraction:
    """Eq. (7): occurrences in s of the k-mers s shares with t, over |s|-k+1."""
    ws, wt = windows(s, k), set(windows(t, k))
    return Fraction(sum(1 for w in ws if w in wt), len(ws))


def brute_filtered(rows, cols, k, theta, tau):
    def cand(a, b):
        if brute_summin(a, b, k) < 1:
            return False
        th = Fraction(*theta)
        if theta[0] and (len(a) < th * len(b) or len(b) < th * len(a)):
            return False
        ta = Fraction(*tau)
        if tau[0] and (brute_p(a, b, k) < ta or brute_p(b, a, k) < ta):
            return False
        return True

    def bh(q, targets, q_is_row):
        vals = {}
        for t, g in enumerate(targets):
            if cand(q, g) if q_is_row else cand(g, q):
                vals[t] = Fraction(brute_summin(q, g, k), brute_summax(q, g, k))
        if not vals:
            return []
        m = max(vals.values())
        return sorted(t for t, v in vals.items() if v == m)

    row_bh = [bh(a, cols, True) for a in rows]
    col_bh = [bh(b, rows, False) for b in cols]
    return row_bh, col_bh, [(a, b) for a in range(len(rows)) for b in row_bh[a] if a in col_bh[b]]


def test_hand_worked():
    # k=2.  a = ACDEFGHIK (8 windows).  b1 = ACDEFGHIKLMNPQRST: shares all 8
    # windows (GJ 8/16), but |a| / |b1| = 9/17 < 0.6.  b2 = ACDEWWW shares
    # AC CD DE (GJ 3/11), lengths 9 and 7.
    rows, cols = [b"ACDEFGHIK"], [b"ACDEFGHIKLMNPQRST", b"ACDEWWW"]
    ds = synth.from_strings([rows, cols])
    assert oracle.filtered_pair(ds, 0, 1, 2)[0] == [[0]]                    # no filter: b1 wins
    assert oracle.filtered_pair(ds, 0, 1, 2, theta=(3, 5))[0] == [[1]]      # theta 0.6 drops b1
    # tau: p(a -> b2) = 3/8 and p(b2 -> a) = 3/6, so tau = 0.4 drops b2 (3/8 < 0.4) ...
    assert oracle.filtered_pair(ds, 0, 1, 2, theta=(3, 5), tau=(2, 5))[0] == [[]]
    # ... while tau = 3/8 keeps it
    assert oracle.filtered_pair(ds, 0, 1, 2, theta=(3, 5), tau=(3, 8))[0] == [[1]]


@pytest.mark.parametrize("seed", range(6))
def test_brute_force(seed):
    ds = synth.random_tiny(500 + seed, n_genomes=2, max_genes=6, max_len=24, letters=b"ACDE")
    rows = [ds.gene(g) for g in range(ds.genome_ptr[0], ds.genome_ptr[1])]
    cols = [ds.gene(g) for g in range(ds.genome_ptr[1], ds.genome_ptr[2])]
    for k, theta, tau in [(2, (0, 1), (1, 2)), (2, (2, 3), (0, 1)), (3, (1, 2), (1, 3)), (1, (4, 5), (3, 4))]:
        got = oracle.filtered_pair(ds, 0, 1, k, theta, tau)
        assert list(got) == list(brute_filtered(rows, cols, k, theta, tau)), (k, theta, tau)
