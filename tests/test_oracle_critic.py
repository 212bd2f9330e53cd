"""Pins of the oracle's critic targets (Sec. II: the partial K-step
cost-to-go stored with V_x for the critic).

* a window covering the whole horizon is the trajectory's total cost, as
  the solver itself accounted it (the final J of a solve);
* K = 1 leaves the knot's own running cost (plus l_T at the last knot);
* adjacent windows telescope: Vbar_k - Vbar_{k+1} = l_k - l_{k+K};
* the terminal knot holds l_T alone, for every K;
* the costs are non-negative, so Vbar grows with K.
"""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W


@pytest.mark.parametrize("make", [W.pointmass, W.planar3, W.arm7, W.dubins])
def test_critic_targets_pins(oracle_mod, make):
    prob = make(seed=3)
    o = oracle_mod.Oracle.from_problem(prob)
    b = W.make_batch(prob, 2, seed=4, T=12)
    r = o.solve(b.x0, b.T, max_iter=4, tol=1e-8)
    for i in range(2):
        T = int(b.T[i])
        X, U = r["X"][i, :T + 1], r["U"][i, :T]
        full = o.critic_targets(X, U, T)
        assert full[0] == pytest.approx(r["J"][i], rel=1e-12)
        l = np.array([o.cost_value(X[k], U[k]) for k in range(T)])
        lT = o.cost_value(X[T], terminal=True)
        one = o.critic_targets(X, U, 1)
        np.testing.assert_allclose(one[:T - 1], l[:T - 1], rtol=1e-14)
        assert one[T - 1] == pytest.approx(l[T - 1] + lT, rel=1e-14)
        for K in (1, 3, 5, T, T + 4):
            v = o.critic_targets(X, U, K)
            assert v[T] == pytest.approx(lT, rel=1e-14)
            for k in range(T - K):
                # both windows end before T: they differ by the knots leaving and entering
                if k + 1 + K <= T - 1:
                    assert v[k] - v[k + 1] == pytest.approx(l[k] - l[k + K], abs=1e-12 * max(v[k], 1.0))
        prev = o.critic_targets(X, U, 1)
        for K in range(2, T + 2):
            cur = o.critic_targets(X, U, K)
            assert np.all(cur >= prev - 1e-12 * np.abs(prev))
            prev = cur
