"""Parity of the rigid-body-tree systems (7-DoF arm, quadruped-shaped floating
base with soft contact and 10 substeps per knot) with the FP64 oracle, under
the oracle's own replayed step sequence; same tolerances and conditioning
rule as the planar cases (see test_gpu_parity.py)."""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W
from test_gpu_parity import _check, _check_consistency, _sensitivity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


def _solver(P, prob, T_max, prec, actor=False):
    s = P.Solver.__new__(P.Solver)
    s.prob = prob
    s.T_max = T_max
    # zero-control warm start unless the actor is asked for
    s.problem = P.tocreate_problem(prob.sys, prob.params, T_max, actor_w=prob.actor_w if actor else None)
    s.opts = P.to_default_opts(prec=prec)
    s.batch = None
    s._cap = (0, 0, P.TO_MIXED)
    return s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_arm7_replay(P, oracle_mod, prec):
    prob = W.arm7(seed=1)
    if prec == "fp64":
        b = W.make_batch(prob, 8, seed=3, T=(20, 60))
        iters = 12
    else:
        # float32 needs well-conditioned replays: short horizons, few
        # iterations (the chain's own rounding noise under the 1e-15 probe is
        # already ~1e-14, so only the best-conditioned instances take the
        # strict bound; the rest take the conditioning-scaled one)
        b = W.make_batch(prob, 16, seed=3, T=(10, 20))
        iters = 3
    o = oracle_mod.Oracle.from_problem(prob)
    ro = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8)
    kappa = _sensitivity(o, b, ro, iters)
    s = _solver(P, prob, 64, P.TO_FP64 if prec == "fp64" else P.TO_MIXED)
    rg = s.solve(b.x0, b.T, forced_alpha=ro["alpha_hist"], max_iter=iters)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.sum() >= 2
    _check_consistency(o, b, rg, prec, min_checked=4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("lanes", [64, 32])
def test_quad_replay(P, oracle_mod, prec, lanes):
    # six short replays: the oracle's sensitivity to a 1e-15 move of x0 is
    # 4e-15 .. 6e-14 here, so at least two instances take the strict mixed
    # bounds (kappa < 1e-14) and all take the FP64 one.  Each candidate's
    # partner lane factors its mass matrix: lane c + 32 (the other warp) at
    # 64 lanes, lane c + 16 at 32 lanes, where the 48 tangent directions also
    # take two passes
    prob = W.quad(seed=2, with_actor=False)
    b = W.make_batch(prob, 6, seed=1, T=6)
    o = oracle_mod.Oracle.from_problem(prob)
    ro = o.solve(b.x0, b.T, max_iter=2, tol=1e-8)
    kappa = _sensitivity(o, b, ro, 2)
    s = _solver(P, prob, 8, P.TO_FP64 if prec == "fp64" else P.TO_MIXED)
    rg = s.solve(b.x0, b.T, forced_alpha=ro["alpha_hist"], max_iter=2, group_lanes=lanes, groups_per_block=1)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.sum() >= (6 if prec == "fp64" else 2), kappa
    _check_consistency(o, b, rg, prec, min_checked=4)


def test_quad_warm_start_rollout(P, oracle_mod):
    """max_iter = 0: the zero-control rollout through 10 substeps of contact dynamics."""
    prob = W.quad(seed=3, with_actor=False)
    b = W.make_batch(prob, 4, seed=2, T=20)
    o = oracle_mod.Oracle.from_problem(prob)
    s = _solver(P, prob, 20, P.TO_FP64)
    rg = s.solve(b.x0, b.T, max_iter=0)
    for i in range(4):
        X, J = o.rollout(b.x0[i], np.zeros((20, 12)))
        assert np.abs(rg["X"][i] - X).max() <= 1e-10 * np.abs(X).max()
        assert abs(rg["J"][i] - J) <= 1e-10 * abs(J)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quad_actor_warm_start(P, oracle_mod, prec):
    """S1: the actor MLP (36-256-256-12, tanh) rolled out through the contact
    dynamics gives the initial guess; then two replayed iterations."""
    prob = W.quad(seed=4, with_actor=True)
    b = W.make_batch(prob, 3, seed=5, T=10)
    o = oracle_mod.Oracle.from_problem(prob)
    s = _solver(P, prob, 10, P.TO_FP64 if prec == "fp64" else P.TO_MIXED, actor=True)
    r0 = o.solve(b.x0, b.T, max_iter=1, forced=np.full((3, 1), -1))
    g0 = s.solve(b.x0, b.T, max_iter=0)
    tol = 1e-10 if prec == "fp64" else 1e-4
    for i in range(3):
        assert np.abs(g0["U"][i] - r0["U"][i]).max() <= tol * np.abs(r0["U"][i]).max()
        assert np.abs(g0["X"][i] - r0["X"][i]).max() <= tol * np.abs(r0["X"][i]).max()
    ro = o.solve(b.x0, b.T, max_iter=2, tol=1e-8)
    kappa = _sensitivity(o, b, ro, 2)
    rg = s.solve(b.x0, b.T, forced_alpha=ro["alpha_hist"], max_iter=2)
    _check(ro, rg, kappa, prec, b.T)



@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quad_full_shape_replay(P, oracle_mod, prec):
    """The bench's quadruped workload at full size (B = 2048, T = 100, actor
    warm start, default launch shape: more instances than resident groups, so
    groups refill from the queue).  Four sampled instances replay the oracle's
    first step and are compared element by element (100 knots of stiff
    contact: a 1e-15 move of x0 already moves the oracle's trajectory by
    1e-13 to 1e-11 on these four, so one or two are well conditioned,
    depending on the host's rounding); every other
    instance stops after its warm start, and four of those are compared with
    the oracle's actor rollout."""
    prob = W.quad(seed=0)
    b = W.make_batch(prob, 2048, seed=0, T=100)
    o = oracle_mod.Oracle.from_problem(prob)
    idx = np.array([300, 1400, 1700, 2000])
    sub = W.Batch(b.x0[idx], b.T[idx])
    iters = 1
    ro = o.solve(sub.x0, sub.T, max_iter=iters, tol=1e-8, threads=len(idx))
    kappa = _sensitivity(o, sub, ro, iters)
    forced = np.full((2048, iters), -1, np.int32)
    forced[idx] = ro["alpha_hist"]
    s = _solver(P, prob, 100, P.TO_FP64 if prec == "fp64" else P.TO_MIXED, actor=True)
    rg = s.solve(b.x0, b.T, forced_alpha=forced, max_iter=iters)
    sel = {k: (v[idx] if isinstance(v, np.ndarray) and v.shape[:1] == (2048,) else v) for k, v in rg.items()}
    well = _check(ro, sel, kappa, prec, sub.T)
    if prec == "fp64":
        assert well.sum() >= 1, kappa
    _check_consistency(o, sub, sel, prec, min_checked=2)
    # instances that stopped at the warm start: the actor's rollout
    other = np.array([1, 701, 1401, 2046])
    r0 = o.solve(b.x0[other], b.T[other], max_iter=1, forced=np.full((4, 1), -1), threads=4)
    tol = 1e-10 if prec == "fp64" else 1e-4
    for k, i in enumerate(other):
        assert rg["iters"][i] == 0
        assert np.abs(rg["X"][i] - r0["X"][k]).max() <= tol * np.abs(r0["X"][k]).max()
        assert abs(rg["J"][i] - r0["J"][k]) <= tol * abs(r0["J"][k])
