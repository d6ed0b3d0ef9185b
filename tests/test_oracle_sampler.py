"""Pins of the oracle's row sampler (uniform sampling without replacement, Algorithm 2)."""
from pathlib import Path

import numpy as np

GOLD = Path(__file__).parent / "golden" / "splitmix64_seed1234567.txt"


def _golden():
    return [int(l) for l in GOLD.read_text().splitlines() if l.strip() and not l.startswith("#")]


def test_splitmix64_published_outputs(oracle_lib):
    ref = _golden()
    assert [oracle_lib.key(1234567, i) for i in range(len(ref))] == ref


def test_keys_distinct(oracle_lib):
    keys = {oracle_lib.key(99, q) for q in range(20000)}
    assert len(keys) == 20000


def test_sample_is_m_smallest_keys_brute_force(oracle_lib):
    for seed, Q, m in [(1, 50, 7), (2, 64, 64), (3, 33, 1), (4, 100, 99), (5, 10, 20)]:
        idx = oracle_lib.sample(seed, Q, m)
        keys = np.array([oracle_lib.key(seed, q) for q in range(Q)], dtype=np.uint64)
        brute = np.sort(np.argsort(keys, kind="stable")[:min(m, Q)])
        assert np.array_equal(idx, brute)
        assert np.all(np.diff(idx) > 0) and idx.min() >= 0 and idx.max() < Q


def test_sample_uniform_inclusion(oracle_lib):
    """Every row is included with probability m/Q: chi-square over 3000 seeds."""
    Q, m, S = 40, 10, 3000
    counts = np.zeros(Q)
    for s in range(S):
        counts[oracle_lib.sample(1000 + s, Q, m)] += 1
    expect = S * m / Q
    var = S * (m / Q) * (1 - m / Q)
    chi2 = np.sum((counts - expect) ** 2 / var)
    assert chi2 < Q + 6 * np.sqrt(2 * Q)        # ~ chi2(Q) well inside its tail
    # pairs: rows 0 and 1 together with probability m(m-1)/(Q(Q-1))
    both = sum(1 for s in range(S) if {0, 1} <= set(oracle_lib.sample(1000 + s, Q, m)))
    pe = m * (m - 1) / (Q * (Q - 1))
    assert abs(both / S - pe) < 5 * np.sqrt(pe * (1 - pe) / S)
