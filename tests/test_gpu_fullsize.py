"""Parity at the benchmark's size (50 genomes x ~3000 genes, k=6), in the
launch configuration bench.py times: the whole result recomputed by oracle B
(every genome pair), a sampled genome pair by oracle A, and properties that
hold at any size on the whole result."""
import pytest

from tests._fullsize import check_properties, check_sampled_pair, check_whole_against_oracle_b, run_full

pytestmark = pytest.mark.gpu

SAMPLED_PAIRS = [(17, 42)]


@pytest.fixture(scope="module")
def full():
    return run_full("pan50x3000", expect_k=6)


@pytest.mark.parametrize("gi,gj", SAMPLED_PAIRS)
def test_sampled_pairs_against_oracle(full, gi, gj):
    check_sampled_pair(full, gi, gj)


def test_whole_result_against_oracle_b(full):
    check_whole_against_oracle_b(full)


def test_properties_at_full_size(full):
    check_properties(full)
