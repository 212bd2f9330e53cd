"""The GPU ranking (torank_candidates) against the oracle: float32 scores
within 1e-5 of the float64 network, and a selection that is valid for the
float64 scores up to that rounding (every chosen candidate scores at least
the N-th largest minus the tolerance, every other at most plus it), exact
where no score lies within the tolerance of the threshold."""
import numpy as np
import pytest

import oracle
from paper_2602_19699_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


@pytest.mark.parametrize("make,N", [(W.planar3, 64), (W.planar3, 1000), (W.arm7, 500), (W.quad, 100), (W.dubins, 3)])
def test_ranking_matches_oracle(P, make, N):
    prob = make(seed=2)
    Cn = 10 * N + 37                                  # a ragged last tile
    X = W.make_batch(prob, Cn, seed=9).x0
    w = W.std_critic_weights(prob.n, seed=5)
    r = P.Ranker(prob.n, w)
    idx, sc = r.rank(X, N, want_scores=True)
    ref_idx, s = oracle.rank_candidates(w, X, N)
    np.testing.assert_allclose(sc, s, rtol=1e-5)
    assert np.all(np.diff(idx) > 0) and idx.size == N
    thr = np.sort(s)[::-1][N - 1]
    tol = 1e-5 * thr
    chosen = np.zeros(Cn, bool)
    chosen[idx] = True
    assert np.all(s[chosen] >= thr - tol)
    assert np.all(s[~chosen] <= thr + tol)
    clear = np.abs(s - thr) > tol
    np.testing.assert_array_equal(chosen[clear], np.isin(np.arange(Cn), ref_idx)[clear])
    r.close()


def test_ranking_ties_take_lower_indices(P):
    w = W.std_critic_weights(4, seed=1)
    X = np.tile(np.random.default_rng(0).normal(size=(1, 4)), (50, 1))   # all candidates identical
    r = P.Ranker(4, w)
    np.testing.assert_array_equal(r.rank(X, 7), np.arange(7))
    r.close()
