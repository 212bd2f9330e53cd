"""Pins of the oracle's iLQR against closed forms, brute-force solves and invariants.

* linear-quadratic instance: one iteration at alpha = 1 reproduces the exact
  minimiser of the dense KKT system (numpy's LU), the next gives a zero step;
* horizons <= 5 on every system: the Riccati step equals the minimiser of the
  dense LQ subproblem built from the (numpy-)clipped Hessians;
* the cost strictly decreases at every accepted step;
* the line search accepts the smallest j with J(alpha_j) < J_old;
* at convergence the open-loop gradient vanishes and V_x(0) = dJ*/dx0
  (envelope theorem, finite differences over re-solves);
* the actor MLP equals torch's float64 CPU evaluation.
"""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W


def _kkt_solve(A, B, Hx, Hu, gx, gu, x0, T):
    """min sum_k 1/2 x'Hx_k x + 1/2 u'Hu_k u + gx_k'x + gu_k'u (+ terminal at k=T)
    s.t. x_0 = x0, x_{k+1} = A_k x_k + B_k u_k, by a dense solve of the KKT system."""
    n, m = B[0].shape
    nx, nu = (T + 1) * n, T * m
    nv = nx + nu
    H = np.zeros((nv, nv))
    g = np.zeros(nv)
    for k in range(T + 1):
        H[k * n:(k + 1) * n, k * n:(k + 1) * n] = Hx[k]
        g[k * n:(k + 1) * n] = gx[k]
    for k in range(T):
        s = nx + k * m
        H[s:s + m, s:s + m] = Hu[k]
        g[s:s + m] = gu[k]
    nc = (T + 1) * n
    G = np.zeros((nc, nv))
    b = np.zeros(nc)
    G[0:n, 0:n] = np.eye(n)
    b[0:n] = x0
    for k in range(T):
        r = (k + 1) * n
        G[r:r + n, (k + 1) * n:(k + 2) * n] = np.eye(n)
        G[r:r + n, k * n:(k + 1) * n] = -A[k]
        G[r:r + n, nx + k * m:nx + (k + 1) * m] = -B[k]
    K = np.block([[H, G.T], [G, np.zeros((nc, nc))]])
    sol = np.linalg.solve(K, np.concatenate([-g, b]))
    return sol[:nx].reshape(T + 1, n), sol[nx:nv].reshape(T, m)


def test_lq_instance_one_iteration_is_exact(oracle_mod):
    prob = W.pointmass(seed=0, n_bumps=0)
    o = oracle_mod.Oracle.from_problem(prob)
    T = 50
    x0 = np.array([1.5, -0.7, 0.2, 0.1])
    dt, wu, wp, wv = prob.params[0], prob.params[1], prob.params[5], prob.params[6]
    A = np.eye(4); A[0, 2] = A[1, 3] = dt
    Bm = np.zeros((4, 2)); Bm[2, 0] = Bm[3, 1] = dt
    Hx = [np.zeros((4, 4))] * T + [np.diag([2 * wp, 2 * wp, 2 * wv, 2 * wv])]
    Hu = [2 * wu * np.eye(2)] * T
    Xs, Us = _kkt_solve([A] * T, [Bm] * T, Hx, Hu, [np.zeros(4)] * (T + 1), [np.zeros(2)] * T, x0, T)
    forced = np.array([[0, 0] + [-1] * 8])
    r = o.solve(x0, T, max_iter=10, eps=0.0, forced=forced)
    assert r["iters"][0] == 2
    scale = np.abs(Us).max()
    np.testing.assert_allclose(r["U"][0], Us, atol=1e-10 * scale)
    np.testing.assert_allclose(r["X"][0], Xs, atol=1e-10 * np.abs(Xs).max())
    # the second iteration is a zero step
    assert abs(r["J_hist"][0, 2] - r["J_hist"][0, 1]) < 1e-12 * abs(r["J_hist"][0, 1])
    # and the one-iteration result is the same trajectory
    r1 = o.solve(x0, T, max_iter=10, eps=0.0, forced=np.array([[0] + [-1] * 9]))
    np.testing.assert_allclose(r1["U"][0], Us, atol=1e-10 * scale)


def _numpy_clip(Q, eps):
    S, Wm = np.linalg.eigh(Q)
    P = Wm @ np.diag(np.maximum(S, eps)) @ Wm.T
    return 0.5 * (P + P.T)


@pytest.mark.parametrize("sysid", [W.POINTMASS, W.PLANAR3, W.ARM7, W.QUAD, W.DUBINS])
def test_riccati_step_equals_dense_lq_subproblem(oracle_mod, sysid):
    prob = W.make_problem(sysid, seed=21)
    o = oracle_mod.Oracle.from_problem(prob)
    n, m = prob.n, prob.m
    T = 5
    rng = np.random.default_rng(sysid)
    x0 = W.make_batch(prob, 1, seed=3).x0[0]
    U = rng.normal(scale=0.5 if sysid != W.QUAD else 2.0, size=(T, m))
    X, _ = o.rollout(x0, U)
    eps = 1e-8
    K, k, _, rc = o.backward(X, U, eps)
    assert rc == 0
    A, Bm, Hx, Hu, gx, gu = [], [], [], [], [], []
    for t in range(T):
        At, Bt = o.linearize(X[t], U[t])
        _, g, H = o.cost(X[t], U[t])
        A.append(At); Bm.append(Bt)
        Hx.append(_numpy_clip(H[:n, :n], eps)); Hu.append(_numpy_clip(H[n:, n:], eps))
        assert np.abs(H[n:, :n]).max() == 0.0      # l_ux = 0 in every workload
        gx.append(g[:n]); gu.append(g[n:])
    _, g, H = o.cost(X[T], terminal=True)
    Hx.append(_numpy_clip(H, eps)); gx.append(g)
    dX, dU = _kkt_solve(A, Bm, Hx, Hu, gx, gu, np.zeros(n), T)
    # the Riccati policy du = k + K dx applied to the same linear model
    dx = np.zeros(n)
    dU_r = np.zeros((T, m))
    for t in range(T):
        dU_r[t] = k[t] + K[t] @ dx
        dx = A[t] @ dx + Bm[t] @ dU_r[t]
    np.testing.assert_allclose(dU_r, dU, atol=1e-8 * max(1.0, np.abs(dU).max()))


@pytest.mark.parametrize("sysid,B,T", [(W.POINTMASS, 6, 50), (W.PLANAR3, 3, 60), (W.ARM7, 2, 30), (W.QUAD, 1, 20), (W.DUBINS, 6, 60)])
def test_cost_strictly_decreases_and_line_search_rule(oracle_mod, sysid, B, T):
    prob = W.make_problem(sysid, seed=31)
    o = oracle_mod.Oracle.from_problem(prob)
    b = W.make_batch(prob, B, seed=5, T=T)
    max_iter = 30 if sysid != W.QUAD else 6
    r = o.solve(b.x0, b.T, max_iter=max_iter, tol=1e-8)
    for i in range(B):
        it = r["iters"][i]
        assert it >= 1
        Jh = r["J_hist"][i, :it + 1]
        assert np.all(np.diff(Jh) < 0), Jh
        assert abs(Jh[-1] - r["J"][i]) == 0.0
        assert r["status"][i] & 15 in (1, 2, 3)
    # the rule, checked on instance 0's first iteration from the zero-control guess
    x0 = b.x0[0]
    Tn = int(b.T[0])
    U0 = np.zeros((Tn, prob.m)) if prob.actor_w is None else None
    if U0 is not None:
        X0, J0 = o.rollout(x0, U0)
        K, k, _, _ = o.backward(X0, U0)
        j_star = r["alpha_hist"][0, 0]
        for j in range(j_star + 1):
            _, _, Jj = o.forward_pass(X0, U0, K, k, 0.5 ** j)
            assert (Jj < J0) == (j == j_star)
        assert abs(Jj - r["J_hist"][0, 1]) <= 1e-12 * abs(Jj)


def test_forced_alpha_sequence_replays(oracle_mod):
    prob = W.planar3(seed=2)
    o = oracle_mod.Oracle.from_problem(prob)
    b = W.make_batch(prob, 2, seed=1, T=80)
    r = o.solve(b.x0, b.T, max_iter=12, tol=1e-10)
    f = r["alpha_hist"].copy()
    rf = o.solve(b.x0, b.T, max_iter=12, forced=f)
    np.testing.assert_array_equal(rf["iters"], r["iters"])
    np.testing.assert_array_equal(rf["U"], r["U"])
    np.testing.assert_array_equal(rf["J"], r["J"])


def test_stationarity_and_value_gradient_at_convergence(oracle_mod):
    prob = W.pointmass(seed=4)
    o = oracle_mod.Oracle.from_problem(prob)
    T = 40
    x0 = np.array([1.2, 0.8, 0.0, 0.0])
    r = o.solve(x0, T, max_iter=300, tol=1e-15, want_vx=True)
    U = r["U"][0]
    X = r["X"][0]
    rng = np.random.default_rng(0)
    _, J = o.rollout(x0, U)
    # open-loop gradient along random directions vanishes
    U0 = np.zeros_like(U)
    h = 1e-5
    for _ in range(3):
        d = rng.normal(size=U.shape)
        g = (o.rollout(x0, U + h * d)[1] - o.rollout(x0, U - h * d)[1]) / (2 * h)
        g0 = (o.rollout(x0, U0 + h * d)[1] - o.rollout(x0, U0 - h * d)[1]) / (2 * h)
        assert abs(g) < 1e-5 * max(1.0, abs(g0))
    # V_x at knot 0 is the gradient of the optimal cost w.r.t. x0 (envelope theorem)
    Vx0 = r["Vx"][0, 0]
    for i in range(4):
        e = np.zeros(4); e[i] = 1e-5
        rp = o.solve(x0 + e, T, U_init=U[None], max_iter=300, tol=1e-15)
        rm = o.solve(x0 - e, T, U_init=U[None], max_iter=300, tol=1e-15)
        fd = (rp["J"][0] - rm["J"][0]) / 2e-5
        assert abs(fd - Vx0[i]) < 1e-5 * max(1.0, np.abs(Vx0).max())
    # V_x at the last knot is the terminal-cost gradient
    np.testing.assert_allclose(r["Vx"][0, T], o.cost(X[T], terminal=True)[1], rtol=1e-14)


def test_actor_matches_torch_float64():
    torch = pytest.importorskip("torch")
    import oracle
    prob = W.quad(seed=3)
    o = oracle.Oracle.from_problem(prob)
    w = prob.actor_w.astype(np.float64)
    sizes = W.ACTOR_SIZES
    off = 0
    layers = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        Wt = torch.tensor(w[off:off + fo * fi].reshape(fo, fi)); off += fo * fi
        bt = torch.tensor(w[off:off + fo]); off += fo
        layers.append((Wt, bt))
    rng = np.random.default_rng(0)
    for _ in range(4):
        x = rng.normal(size=36)
        h = torch.tensor(x)
        for li, (Wt, bt) in enumerate(layers):
            h = torch.nn.functional.linear(h, Wt, bt)
            if li < 2:
                h = torch.tanh(h)
        np.testing.assert_allclose(o.actor(x), h.numpy(), rtol=1e-12, atol=1e-13)


def test_actor_warm_start_rolls_out_the_policy(oracle_mod):
    prob = W.quad(seed=6)
    o = oracle_mod.Oracle.from_problem(prob)
    b = W.make_batch(prob, 1, seed=2, T=5)
    r = o.solve(b.x0, b.T, max_iter=1, forced=np.array([[-1]]))
    X, U = r["X"][0], r["U"][0]
    assert r["iters"][0] == 0
    for k in range(5):
        np.testing.assert_allclose(U[k], o.actor(X[k]), rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(X[k + 1], o.step(X[k], U[k]), rtol=1e-14, atol=1e-14)
