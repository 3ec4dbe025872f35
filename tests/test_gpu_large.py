"""Parity on the large plain workload: 200 genomes x ~4000 genes (800k genes,
275 M residues, k=7, all 19900 genome pairs in one all-pairs launch).  The
oracle recomputes sampled genome pairs in full; properties that hold at any
size are checked on the whole result."""
import pytest

from tests._fullsize import check_properties, check_sampled_pair, run_full

pytestmark = pytest.mark.gpu

SAMPLED_PAIRS = [(0, 1), (57, 143), (198, 199)]


@pytest.fixture(scope="module")
def full():
    return run_full("pan200x4000", expect_k=7)


@pytest.mark.parametrize("gi,gj", SAMPLED_PAIRS)
def test_sampled_pairs_against_oracle(full, gi, gj):
    check_sampled_pair(full, gi, gj)


def test_properties_at_full_size(full):
    check_properties(full)
