"""The jerk-controlled Dubins car on the GPU against the oracle: the
oracle's step sequence replayed (conditioning rule of test_gpu_parity.py)
and unforced solves that take the same steps."""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W
from test_gpu_parity import FP64_TOL, _check, _check_consistency, _replay, _sensitivity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dubins_replay(P, oracle_mod, prec):
    prob = W.dubins(seed=2)
    b = W.make_batch(prob, 48, seed=3, T=(30, 100))
    o = oracle_mod.Oracle.from_problem(prob)
    iters = 30
    ro = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8)
    kappa = _sensitivity(o, b, ro, iters)
    rg = _replay(P, prob, b, ro, P.TO_FP64 if prec == "fp64" else P.TO_MIXED, iters, T_max=100)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.mean() >= 0.25
    _check_consistency(o, b, rg, prec, min_checked=12)


def test_dubins_unforced_matches_oracle_choices(P, oracle_mod):
    prob = W.dubins(seed=4)
    b = W.make_batch(prob, 64, seed=5, T=60)
    ro = oracle_mod.Oracle.from_problem(prob).solve(b.x0, b.T, max_iter=100, tol=1e-8, n_alpha=16)
    s = P.Solver(prob, T_max=60, prec=P.TO_FP64)
    rg = s.solve(b.x0, b.T, max_iter=100, tol=1e-8)
    same = np.all(rg["alpha_hist"] == ro["alpha_hist"], axis=1) & (rg["iters"] == ro["iters"])
    assert same.mean() >= 0.8, same.mean()
    ej = np.abs(rg["J"] - ro["J"]) / np.abs(ro["J"])
    assert np.median(ej[same]) < FP64_TOL
