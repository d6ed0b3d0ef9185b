"""Pins of the oracle's Algorithm 2 with mixing (Sec. 5: random signs D, fast orthonormal
mixing F over the rows, uniform sampling S)."""
import numpy as np
import pytest
import scipy.linalg

from paper_1907_05884_gb300 import synth


@pytest.fixture(scope="module")
def mix(oracle_lib):
    from oracle import mixing
    return mixing


@pytest.mark.parametrize("N", [1, 2, 4, 8, 64, 256])
def test_fwht_is_the_normalised_hadamard_matrix(mix, N):
    X = np.random.default_rng(N).standard_normal((N, 3))
    ref = scipy.linalg.hadamard(N) @ X / np.sqrt(N)
    assert np.max(np.abs(mix.fwht(X) - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_fwht_is_an_orthogonal_involution(mix):
    X = np.random.default_rng(5).standard_normal((4096, 2))
    Y = mix.fwht(X)
    assert abs(np.linalg.norm(Y) - np.linalg.norm(X)) < 1e-12 * np.linalg.norm(X)
    assert np.max(np.abs(mix.fwht(Y) - X)) < 1e-12


def test_padded_rows(mix):
    assert [mix.padded_rows(q) for q in (1, 2, 3, 4, 5, 1000, 1024, 1025)] == [1, 2, 4, 4, 8, 1024, 1024, 2048]


def test_signs_follow_the_key_and_are_balanced(mix, oracle_lib):
    d = mix.signs(7, 1 << 14)
    assert set(np.unique(d)) == {-1.0, 1.0}
    for q in (0, 1, 2, 100, 16383):
        assert d[q] == (-1.0 if oracle_lib.key(7, q) >= 1 << 63 else 1.0)
    assert abs(d.mean()) < 4 / np.sqrt(d.size)
    # a different seed gives a different, uncorrelated pattern
    e = mix.signs(8, 1 << 14)
    assert abs((d * e).mean()) < 4 / np.sqrt(d.size)


@pytest.fixture(scope="module")
def problem():
    m = synth.random_model((4, 3, 5), (7, 6, 8), seed=61, density=0.8)
    xyz = synth.points(1500, seed=62)
    u, _ = synth.field_values(xyz, synth.field_spec(63, 5), seed=64)
    return m, xyz, u


def test_all_mixed_rows_give_the_full_least_squares(mix, oracle_lib, problem):
    """F D is orthogonal, so with every one of the N mixed rows kept the solution is the plain
    least-squares fit to all Q points."""
    m, xyz, u = problem
    Q = xyz.shape[1]
    N = mix.padded_rows(Q)
    alpha, rc = mix.refit_mixed(m, xyz, u, N, seed_signs=3, seed_rows=4)
    assert rc == 0
    A = oracle_lib.design_matrix(m, xyz, np.arange(Q, dtype=np.int64))
    ref = np.linalg.lstsq(A, u, rcond=None)[0]
    assert np.linalg.norm(alpha.ravel() - ref) < 1e-10 * np.linalg.norm(ref)


def test_mixed_system_is_an_orthogonal_image(mix, oracle_lib, problem):
    m, xyz, u = problem
    A, b = mix.mixed_system(m, xyz, u, seed_signs=9)
    W = oracle_lib.design_matrix(m, xyz, np.arange(xyz.shape[1], dtype=np.int64))
    assert np.max(np.abs(A.T @ A - W.T @ W)) < 1e-10 * np.max(np.abs(W.T @ W))
    assert abs(b @ b - u @ u) < 1e-10 * (u @ u)


def test_noise_free_data_recovered_from_few_mixed_rows(mix, oracle_lib):
    m = synth.random_model((3, 4, 2), (5, 6, 4), seed=71, density=1.0, orthonormal=True)
    xyz = synth.points(2000, seed=72)
    W = oracle_lib.design_matrix(m, xyz, np.arange(2000, dtype=np.int64))
    a_true = np.random.default_rng(73).standard_normal(m.R)
    u = W @ a_true
    alpha, rc = mix.refit_mixed(m, xyz, u, 3 * m.R, seed_signs=74, seed_rows=75)
    assert rc == 0
    assert np.linalg.norm(alpha.ravel() - a_true) < 1e-10 * np.linalg.norm(a_true)


def test_mixing_flattens_the_leverage_scores(mix, oracle_lib):
    """The point of F D (Sec. 5): the row leverage scores of F D W are spread out, so uniform
    sampling sees every direction; on clustered points the largest score drops."""
    m = synth.random_model((4, 4, 4), (7, 7, 7), seed=81, density=1.0, orthonormal=True)
    xyz = synth.points(4096, seed=82, clustered=0.9)
    W = oracle_lib.design_matrix(m, xyz, np.arange(4096, dtype=np.int64))
    A, _ = mix.mixed_system(m, xyz, np.zeros(4096), seed_signs=83)

    def lev(X):
        q, _ = np.linalg.qr(X)
        return np.sum(q * q, axis=1)

    lw, la = lev(W), lev(A)
    assert abs(lw.sum() - m.R) < 1e-8 and abs(la.sum() - m.R) < 1e-8
    assert la.max() < 0.5 * lw.max()
