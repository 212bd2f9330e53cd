"""The Levenberg-Marquardt variant on the GPU (opts.reg = TO_REG_LM) against
the oracle's: the oracle's accepted step sequence replayed (its mu schedule
and backward-pass retries then follow from the same arithmetic), and
unforced point-mass solves that take the same steps."""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W
from test_gpu_parity import FP64_TOL, _check, _inst_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


def _sensitivity_lm(o, b, ro, max_iter):
    x1 = b.x0 * (1 + 1e-15 * np.random.default_rng(1).choice([-1.0, 1.0], size=b.x0.shape))
    r2 = o.solve(x1, b.T, max_iter=max_iter, forced=ro["alpha_hist"], reg="lm")
    k = _inst_rel(r2["X"], ro["X"], b.T)
    k[~np.isfinite(k)] = np.inf
    return k


@pytest.mark.parametrize("lanes", [8, 32])       # sub-warp groups, and a whole warp (the lane-parallel factor)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_planar3_lm_replay(P, oracle_mod, prec, lanes):
    prob = W.planar3(seed=1)
    b = W.make_batch(prob, 24, seed=2, T=(20, 40))
    o = oracle_mod.Oracle.from_problem(prob)
    iters = 8
    ro = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8, n_alpha=16, reg="lm")
    kappa = _sensitivity_lm(o, b, ro, iters)
    s = P.Solver(prob, T_max=40, prec=P.TO_FP64 if prec == "fp64" else P.TO_MIXED, reg=P.TO_REG_LM,
                 group_lanes=lanes, groups_per_block=64 // lanes)
    rg = s.solve(b.x0, b.T, forced_alpha=ro["alpha_hist"], max_iter=iters)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.sum() >= 4


def test_pointmass_lm_unforced_matches_oracle(P, oracle_mod):
    prob = W.pointmass(seed=3)
    b = W.make_batch(prob, 64, seed=4)
    ro = oracle_mod.Oracle.from_problem(prob).solve(b.x0, b.T, max_iter=100, tol=1e-8, n_alpha=16, reg="lm")
    s = P.Solver(prob, T_max=50, prec=P.TO_FP64, reg=P.TO_REG_LM)
    rg = s.solve(b.x0, b.T, max_iter=100, tol=1e-8)
    same = np.all(rg["alpha_hist"] == ro["alpha_hist"], axis=1) & (rg["iters"] == ro["iters"])
    assert same.mean() >= 0.95, same.mean()
    ej = np.abs(rg["J"] - ro["J"]) / np.abs(ro["J"])
    assert ej[same].max() < FP64_TOL
    np.testing.assert_array_equal(rg["status"][same], ro["status"][same])
