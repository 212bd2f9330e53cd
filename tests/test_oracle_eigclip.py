"""Pins of the eigenvalue clipping (Sec. IV-B) against numpy's symmetric eigensolver."""
import numpy as np
import pytest


def _numpy_clip(Q, eps):
    S, Wm = np.linalg.eigh(Q)
    P = Wm @ np.diag(np.maximum(S, eps)) @ Wm.T
    return 0.5 * (P + P.T)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 14, 36])
def test_clip_matches_library_eigendecomposition(oracle_mod, n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    Q = A + A.T
    eps = 1e-3
    out = oracle_mod.eigclip(Q, eps)
    np.testing.assert_allclose(out, _numpy_clip(Q, eps), atol=1e-12 * max(1, np.abs(Q).max()))
    assert np.linalg.eigvalsh(out).min() >= eps * (1 - 1e-9)
    S, Wm = oracle_mod.eig(Q)
    np.testing.assert_allclose(np.sort(S), np.linalg.eigvalsh(Q), atol=1e-12 * np.abs(Q).max())
    np.testing.assert_allclose(Wm.T @ Wm, np.eye(n), atol=1e-12)


def test_clip_is_identity_on_positive_definite_input(oracle_mod):
    rng = np.random.default_rng(0)
    A = rng.normal(size=(6, 6))
    Q = A @ A.T + 0.5 * np.eye(6)
    np.testing.assert_allclose(oracle_mod.eigclip(Q, 1e-8), Q, atol=1e-13 * np.abs(Q).max())


def test_full_clip_equals_block_clip_plus_eps(oracle_mod):
    """A Hessian supported on one block: the full-matrix clip equals the clip of
    the block, with eps on the remaining diagonal (those eigenpairs are (0, e_i))."""
    rng = np.random.default_rng(1)
    n, idx = 8, [1, 4, 6]
    A = rng.normal(size=(3, 3))
    blk = A + A.T
    Q = np.zeros((n, n))
    Q[np.ix_(idx, idx)] = blk
    eps = 1e-8
    full = oracle_mod.eigclip(Q, eps)
    expect = np.diag(np.full(n, eps))
    expect[np.ix_(idx, idx)] = _numpy_clip(blk, eps)
    np.testing.assert_allclose(full, expect, atol=1e-13)


def test_zero_matrix_clips_to_eps_identity(oracle_mod):
    np.testing.assert_allclose(oracle_mod.eigclip(np.zeros((4, 4)), 0.25), 0.25 * np.eye(4), atol=0)


def test_guarded_cholesky(oracle_mod):
    rng = np.random.default_rng(2)
    A = rng.normal(size=(5, 5))
    Q = A @ A.T + np.eye(5)
    b = rng.normal(size=5)
    x, rc = oracle_mod.chol_solve(Q, b)
    assert rc == 0
    np.testing.assert_allclose(Q @ x, b, atol=1e-12)
    # indefinite: the pivot test fails and mu I is added until it passes
    Qi = np.diag([1.0, -0.5, 2.0])
    x, rc = oracle_mod.chol_solve(Qi, np.ones(3))
    assert rc == 1
    assert np.all(np.isfinite(x))
