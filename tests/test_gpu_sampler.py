"""Bit-exact parity of the GPU row sampler (fst_sample_rows) with the oracle's sampler
(uniform sampling without replacement, Algorithm 2)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


@pytest.mark.parametrize("seed,Q,m", [(1, 1, 1), (2, 10, 3), (3, 1000, 999), (4, 4096, 1),
                                      (5, 100_003, 4096), (6, 1 << 20, 13_824), (7, 50, 50), (8, 50, 80)])
def test_sampler_matches_oracle(F, oracle_lib, seed, Q, m):
    got = F.sample_rows(seed, Q, m).cpu().numpy()
    ref = oracle_lib.sample(seed, Q, m)
    assert np.array_equal(got, ref)


def test_sampler_full_size(F, oracle_lib):
    """2^24 rows, m = 8 * 24^3 = 110,592 (the refit sample of the 16M-point workload)."""
    seed, Q, m = 0x5EED, 1 << 24, 8 * 24 ** 3
    got = F.sample_rows(seed, Q, m).cpu().numpy()
    ref = oracle_lib.sample(seed, Q, m)
    assert np.array_equal(got, ref)


def test_sampler_zero_sizes(F):
    assert F.sample_rows(1, 10, 0).numel() == 0
