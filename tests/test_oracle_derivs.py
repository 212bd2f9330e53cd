"""Pins of the oracle's exact (dual-number) derivatives against central finite differences."""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W


def _state(prob, rng):
    b = W.make_batch(prob, 1, seed=int(rng.integers(1000)))
    x = b.x0[0].copy()
    x[prob.n // 2 if prob.sys != W.POINTMASS else 2:] += rng.normal(scale=0.5, size=prob.n - (prob.n // 2 if prob.sys != W.POINTMASS else 2))
    u = rng.normal(scale=1.0, size=prob.m)
    return x, u


def _rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("sysid", [W.POINTMASS, W.PLANAR3, W.ARM7, W.QUAD, W.DUBINS])
def test_dynamics_jacobians_match_central_differences(oracle_mod, sysid):
    prob = W.make_problem(sysid, seed=11)
    o = oracle_mod.Oracle.from_problem(prob)
    rng = np.random.default_rng(sysid)
    for _ in range(2):
        x, u = _state(prob, rng)
        A, B = o.linearize(x, u)
        Afd = np.zeros_like(A)
        Bfd = np.zeros_like(B)
        for j in range(prob.n):
            h = 1e-6 * max(1.0, abs(x[j]))
            e = np.zeros(prob.n); e[j] = h
            Afd[:, j] = (o.step(x + e, u) - o.step(x - e, u)) / (2 * h)
        for j in range(prob.m):
            h = 1e-6 * max(1.0, abs(u[j]))
            e = np.zeros(prob.m); e[j] = h
            Bfd[:, j] = (o.step(x, u + e) - o.step(x, u - e)) / (2 * h)
        assert _rel(A, Afd) < 1e-7
        assert _rel(B, Bfd) < 1e-7


@pytest.mark.parametrize("sysid", [W.POINTMASS, W.PLANAR3, W.ARM7, W.QUAD, W.DUBINS])
@pytest.mark.parametrize("terminal", [False, True])
def test_cost_gradient_and_hessian_match_central_differences(oracle_mod, sysid, terminal):
    prob = W.make_problem(sysid, seed=12)
    o = oracle_mod.Oracle.from_problem(prob)
    rng = np.random.default_rng(100 + sysid)
    x, u = _state(prob, rng)
    if sysid == W.POINTMASS:
        # sit on a bump so that the Gaussian terms are active
        x[0:2] = prob.meta["centres"][0] + 0.05
    l, g, H = o.cost(x, u, terminal=terminal)
    z = x if terminal else np.concatenate([x, u])
    nz = z.size

    def f(zz):
        return o.cost_value(zz[:prob.n], None if terminal else zz[prob.n:], terminal=terminal)

    def grad(zz):
        return o.cost(zz[:prob.n], None if terminal else zz[prob.n:], terminal=terminal)[1]

    assert abs(f(z) - l) < 1e-14 * max(1, abs(l))
    gfd = np.zeros(nz)
    Hfd = np.zeros((nz, nz))
    for j in range(nz):
        h = 1e-6 * max(1.0, abs(z[j]))
        e = np.zeros(nz); e[j] = h
        gfd[j] = (f(z + e) - f(z - e)) / (2 * h)
        Hfd[:, j] = (grad(z + e) - grad(z - e)) / (2 * h)
    assert _rel(g, gfd) < 1e-7
    assert _rel(H, Hfd) < 1e-7
    np.testing.assert_allclose(H, H.T, atol=1e-12 * max(1, np.abs(H).max()))


def test_contact_jacobian_in_the_softplus_region(oracle_mod):
    """Feet within a few millimetres of the ground, where the softplus bends (beta z ~ 1)."""
    prob = W.quad(seed=13, with_actor=False)
    o = oracle_mod.Oracle(W.QUAD, prob.params)
    th = prob.meta["theta"]
    x = np.zeros(36)
    x[2] = prob.meta["z_nom"] + 0.004
    x[6:18] = np.tile([0.0, th, -2 * th], 4)
    x[18:] = np.random.default_rng(0).normal(scale=0.1, size=18)
    u = np.zeros(12)
    A, B = o.linearize(x, u)
    Afd = np.zeros_like(A)
    for j in range(36):
        h = 1e-6 * max(1.0, abs(x[j]))
        e = np.zeros(36); e[j] = h
        Afd[:, j] = (o.step(x + e, u) - o.step(x - e, u)) / (2 * h)
    assert _rel(A, Afd) < 1e-7
