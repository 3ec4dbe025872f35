"""Parity on the large plain workload: 200 genomes x ~4000 genes (800k genes,
275 M residues, k=7, all 19900 genome pairs in one all-pairs launch).  Oracle B
recomputes the whole result (every genome pair), oracle A a sampled genome
pair in full; properties that hold at any size are checked on the whole
result."""
import pytest

from tests._fullsize import check_properties, check_sampled_pair, check_whole_against_oracle_b, run_full

pytestmark = pytest.mark.gpu

SAMPLED_PAIRS = [(57, 143)]


@pytest.fixture(scope="module")
def full():
    return run_full("pan200x4000", expect_k=7)


@pytest.mark.parametrize("gi,gj", SAMPLED_PAIRS)
def test_sampled_pairs_against_oracle(full, gi, gj):
    check_sampled_pair(full, gi, gj)


def test_whole_result_against_oracle_b(full):
    check_whole_against_oracle_b(full)


def test_properties_at_full_size(full):
    check_properties(full)
