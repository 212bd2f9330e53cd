"""The regularisation guard of the Q_uu Cholesky on the GPU (Sec. IV-B's
mu I, used only when the pivot test fails), against the oracle.

Workload: the Dubins car with a nearly free heading control and a stiff
terminal acceleration weight (w_u = 1e-6, w_aT = 1e9).  The heading is absent
from the terminal cost and, at rest, from every knot's value Hessian, so the
omega pivot of Q_uu = l_uu + B^T V B is about 2 w_u = 2e-6, while the jerk
pivot is about dt^2 2 w_aT = 5e6.  The pivot test d_j > 1e-12 max|diag| then
fails (2e-6 < 5e-6) and mu I is added with mu = 1e-6 max|diag| = 5: every knot
of the first iteration, and the last knot of every later one, is regularised.
The omega gains are -Q_u / (2e-6 + mu), so a wrong mu schedule (or gains
taken from the unshifted factor) changes them by orders of magnitude.

Both sides replay the oracle's accepted step sequence; X, U and the final
gains K are compared element by element on the instances whose replay is well
conditioned (the oracle itself moves by less than 1e-12 when x0 moves by
1e-15), and both set TO_ST_FLAG_REG.  The replay is the first iteration,
where every knot is regularised whatever the rounding; in FP64 the gains of
the backward pass at the new iterate (where the last knot is regularised)
are compared too.  The replay runs with 8-lane groups (the sub-warp
factor, on every lane) and with whole-warp groups (the factor spread over
the warp's lanes, one lower-triangle entry per lane).

Tolerances.  Whenever the guard fires, the failing pivot is far below mu, so
Q_uu + mu I has a condition number of about max|diag| / mu = 1e6 (the shift
rule fixes it).  A float64 solve of it differs between two correct
implementations by up to ~4 kappa 2^-52 ~ 1e-9 (instead of the 1e-10 of the
other FP64 parity tests).  In mixed precision the bound is 5e-2: the pivot
test can only fail for a pivot 1e12 below the largest, so this problem's
value Hessian spans the acceleration weight dt^2 w_aT ~ 5e6 down to the
velocity weight 2, 22 bits apart, and the float32 Riccati products carry the
velocity terms to a couple of significant bits (measured: 0.4 to 1.8 % on
every instance; solving the regularised knots' gains with the float64
factor changed nothing, so the solve is not the limit).
"""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W
from test_gpu_parity import _inst_rel

pytestmark = pytest.mark.gpu

FLAG_REG = 16
KAPPA_SHIFTED = 1e6                                      # max|diag| / mu
GUARD_FP64_TOL = 4 * KAPPA_SHIFTED * 2.0 ** -52 * 2      # ~1.8e-9
GUARD_MIXED_TOL = 5e-2


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


def _problem():
    prob = W.dubins(seed=2)
    prob.params = prob.params.copy()
    prob.params[1] = 1e-6                      # control weight w_u
    prob.params[7 + 2 * 3] = 1e9               # terminal acceleration weight w_aT (3 bumps)
    return prob


def _oracle_replay(o, b, iters, forced, want_K):
    """the oracle's replay of a step sequence, and its sensitivity to x0 * (1 +- 1e-15)"""
    r1 = o.solve(b.x0, b.T, max_iter=iters, forced=forced, want_K=want_K)
    x1 = b.x0 * (1 + 1e-15 * np.random.default_rng(1).choice([-1.0, 1.0], size=b.x0.shape))
    r2 = o.solve(x1, b.T, max_iter=iters, forced=forced, want_K=want_K)
    kx = _inst_rel(r2["X"], r1["X"], b.T)
    kk = _inst_rel(r2["K"], r1["K"], b.T, 0) if want_K else np.zeros_like(kx)
    return r1, kx, kk


@pytest.mark.parametrize("lanes", [8, 32])       # sub-warp groups, and a whole warp (the lane-parallel factor)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_guard_replay(P, oracle_mod, prec, lanes):
    prob = _problem()
    b = W.make_batch(prob, 16, seed=3, T=(20, 40))
    o = oracle_mod.Oracle.from_problem(prob)
    iters = 1                          # the first iteration: every knot is regularised
    ro0 = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8, n_alpha=16)
    assert np.all(ro0["status"] & FLAG_REG)
    fp64 = prec == "fp64"
    ro, kx, kk = _oracle_replay(o, b, iters, ro0["alpha_hist"], want_K=fp64)
    assert np.all(ro["status"] & FLAG_REG)
    s = P.Solver(prob, T_max=40, prec=P.TO_FP64 if fp64 else P.TO_MIXED, group_lanes=lanes,
                 groups_per_block=64 // lanes)
    want = ("X", "U", "K") if fp64 else ("X", "U")
    rg = s.solve(b.x0, b.T, forced_alpha=ro0["alpha_hist"], max_iter=iters, want_vx=1 if fp64 else 0, want=want)
    np.testing.assert_array_equal(rg["iters"], ro["iters"])
    np.testing.assert_array_equal(rg["status"], ro["status"])
    assert np.all(rg["status"] & FLAG_REG)
    well = (kx < 1e-12) & (kk < 1e-11)
    assert well.sum() >= 6, (kx, kk)
    ex = np.maximum(_inst_rel(rg["X"], ro["X"], b.T), _inst_rel(rg["U"], ro["U"], b.T, 0))
    ej = np.abs(rg["J"] - ro["J"]) / np.abs(ro["J"])
    tol = GUARD_FP64_TOL if fp64 else GUARD_MIXED_TOL
    assert ex[well].max() < tol, ex[well]
    assert ej[well].max() < tol, ej[well]
    if fp64:
        # the final backward pass's gains; the last knot's omega row is
        # -Q_ux / (2e-6 + mu) with mu = 5, so it pins the shift
        ek = _inst_rel(rg["K"], ro["K"], b.T, 0)
        assert ek[well].max() < GUARD_FP64_TOL, ek[well]
        for i in np.where(well)[0]:
            T = int(b.T[i])
            Kg, Ko = rg["K"][i, T - 1, 0], ro["K"][i, T - 1, 0]
            assert np.abs(Kg - Ko).max() <= GUARD_FP64_TOL * max(np.abs(Ko).max(), 1e-300)
