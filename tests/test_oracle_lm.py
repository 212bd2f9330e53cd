"""Pins of the oracle's Levenberg-Marquardt variant (Sec. IV-B: the
standard regularisation the paper replaces on the GPU).

* on a linear-quadratic instance, one LM iteration from zero controls is the
  exact minimiser of the dense KKT system whose control Hessian carries the
  first mu (Q_uu + mu I at every knot is that problem's Riccati recursion);
* at LM's fixed point the regulariser drops out: the iteration converges to
  the unregularised KKT optimum;
* every accepted step strictly decreases the cost.
"""
import numpy as np

from paper_2602_19699_gb300 import workload as W
from test_oracle_ilqr import _kkt_solve

MU0 = 1e-6


def _lq(oracle_mod):
    prob = W.pointmass(seed=0, n_bumps=0)
    o = oracle_mod.Oracle.from_problem(prob)
    T = 50
    x0 = np.array([1.5, -0.7, 0.2, 0.1])
    dt, wu, wp, wv = prob.params[0], prob.params[1], prob.params[5], prob.params[6]
    A = np.eye(4); A[0, 2] = A[1, 3] = dt
    Bm = np.zeros((4, 2)); Bm[2, 0] = Bm[3, 1] = dt
    Hx = [np.zeros((4, 4))] * T + [np.diag([2 * wp, 2 * wp, 2 * wv, 2 * wv])]
    Hu = 2 * wu * np.eye(2)
    return o, T, x0, A, Bm, Hx, Hu


def test_one_lm_iteration_is_the_shifted_kkt_solution(oracle_mod):
    o, T, x0, A, Bm, Hx, Hu = _lq(oracle_mod)
    Xs, Us = _kkt_solve([A] * T, [Bm] * T, Hx, [Hu + MU0 * np.eye(2)] * T, [np.zeros(4)] * (T + 1),
                        [np.zeros(2)] * T, x0, T)
    r = o.solve(x0, T, max_iter=10, forced=np.array([[0] + [-1] * 9]), reg="lm")
    assert r["iters"][0] == 1
    np.testing.assert_allclose(r["U"][0], Us, atol=1e-10 * np.abs(Us).max())
    np.testing.assert_allclose(r["X"][0], Xs, atol=1e-10 * np.abs(Xs).max())


def test_lm_converges_to_the_unregularised_optimum(oracle_mod):
    o, T, x0, A, Bm, Hx, Hu = _lq(oracle_mod)
    Xs, Us = _kkt_solve([A] * T, [Bm] * T, Hx, [Hu] * T, [np.zeros(4)] * (T + 1), [np.zeros(2)] * T, x0, T)
    r = o.solve(x0, T, max_iter=100, tol=1e-14, reg="lm")
    np.testing.assert_allclose(r["U"][0], Us, atol=1e-7 * np.abs(Us).max())
    Jstar = o.rollout(x0, Us)[1]
    assert abs(r["J"][0] - Jstar) <= 1e-10 * Jstar


def test_lm_accepted_steps_decrease_the_cost(oracle_mod):
    prob = W.planar3(seed=2)
    o = oracle_mod.Oracle.from_problem(prob)
    b = W.make_batch(prob, 6, seed=3, T=(20, 60))
    r = o.solve(b.x0, b.T, max_iter=40, reg="lm", n_alpha=16)
    for i in range(6):
        h = r["J_hist"][i, :r["iters"][i] + 1]
        assert np.all(np.diff(h) < 0)
    assert np.all(np.isin(r["status"] & 15, [1, 2, 3]))
