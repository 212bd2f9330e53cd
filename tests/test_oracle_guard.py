"""Pins of the regularisation guard of the Q_uu Cholesky (Sec. IV-B: the
Levenberg-Marquardt term mu I, here used only when the plain factor fails).

The rule: the factor of Q_uu is accepted when every pivot d_j (the square of
the Cholesky diagonal) exceeds delta = 1e-12 max|diag Q_uu|; otherwise mu I is
added with mu = 1e-6 max|diag Q_uu|, growing x10, until the pivots of
Q_uu + mu I pass the same test, and the gains solve that shifted system.

The expected shift is found here without the oracle's factor: the pivots of a
symmetric matrix are ratios of consecutive leading principal minors,
d_j = det(A[:j+1, :j+1]) / det(A[:j, :j]), and the solution comes from
numpy's LU solve of (Q_uu + mu* I) x = b.
"""
import numpy as np
import pytest


def _pivots(A):
    """Cholesky pivots of a symmetric matrix as ratios of leading minors."""
    n = A.shape[0]
    dets = [1.0] + [np.linalg.det(A[:j + 1, :j + 1]) for j in range(n)]
    return np.array([dets[j + 1] / dets[j] if dets[j] > 0 else -np.inf for j in range(n)])


def _expected_shift(Q):
    """0 when the plain factor passes the pivot test, else the smallest
    1e-6 mx 10^k (k < 40) whose shifted matrix passes it."""
    mx = np.abs(np.diag(Q)).max()
    delta = 1e-12 * mx
    if np.all(_pivots(Q) > delta):
        return 0.0
    mu = 1e-6 * mx
    for _ in range(40):
        if np.all(_pivots(Q + mu * np.eye(Q.shape[0])) > delta):
            # the shifted matrix is positive definite: numpy's factor exists
            np.linalg.cholesky(Q + mu * np.eye(Q.shape[0]))
            return mu
        mu *= 10.0
    raise AssertionError("no shift found")


def _check(oracle_mod, Q, b, rc_expected, mu_expected=None):
    x, rc = oracle_mod.chol_solve(Q, b)
    assert rc == rc_expected
    mu = _expected_shift(Q)
    if mu_expected is not None:
        assert mu == pytest.approx(mu_expected, rel=1e-12)
    assert (mu > 0) == (rc == 1)
    xs = np.linalg.solve(Q + mu * np.eye(Q.shape[0]), b)
    np.testing.assert_allclose(x, xs, rtol=1e-9, atol=1e-12 * np.abs(xs).max())
    return mu


def test_indefinite_diagonal_exact_shift(oracle_mod):
    # d = (1, -0.5, 2): mx = 2, shifts 2e-6 ... 0.2 leave -0.5 + mu <= 0; 2.0 passes
    Q = np.diag([1.0, -0.5, 2.0])
    b = np.array([1.0, 2.0, 3.0])
    _check(oracle_mod, Q, b, 1, mu_expected=2.0)
    x, _ = oracle_mod.chol_solve(Q, b)
    np.testing.assert_allclose(x, b / np.array([3.0, 1.5, 4.0]), rtol=1e-14)


def test_singular_psd_takes_the_first_shift(oracle_mod):
    rng = np.random.default_rng(3)
    V = rng.normal(size=(4, 2))
    Q = V @ V.T                                     # rank 2: the third pivot is 0
    b = Q @ rng.normal(size=4)                      # a right-hand side in the range
    mx = np.abs(np.diag(Q)).max()
    _check(oracle_mod, Q, b, 1, mu_expected=1e-6 * mx)


def test_pivot_threshold_is_relative_1e_12(oracle_mod):
    b = np.array([1.0, 1.0])
    # a pivot of 5e-13 mx fails the test (mu = 1e-6 added); 2e-12 mx passes it
    _check(oracle_mod, np.diag([1.0, 5e-13]), b, 1, mu_expected=1e-6)
    _check(oracle_mod, np.diag([1.0, 2e-12]), b, 0, mu_expected=0.0)
    # the threshold scales with max|diag|
    _check(oracle_mod, np.diag([1e6, 5e-7]), b, 1, mu_expected=1.0)
    _check(oracle_mod, np.diag([1e6, 2e-6]), b, 0, mu_expected=0.0)


@pytest.mark.parametrize("seed", range(6))
def test_random_indefinite_matrices(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(2, 8))
    A = rng.normal(size=(m, m))
    S = np.diag(rng.uniform(-1.0, 3.0, size=m))
    Q = A @ S @ A.T                                 # indefinite in general
    b = rng.normal(size=m)
    mu = _expected_shift(Q)
    _check(oracle_mod, Q, b, 1 if mu > 0 else 0)


def test_unusable_matrices_fail(oracle_mod):
    for Q in (np.zeros((3, 3)), np.diag([1.0, np.nan, 1.0]), np.diag([-1.0, -2.0])):
        _, rc = oracle_mod.chol_solve(Q, np.ones(Q.shape[0]))
        if np.all(np.diag(Q) < 0):
            # max|diag| > 0: shifts up to 1e33 mx make it positive definite
            assert rc == 1
        else:
            assert rc == -1
