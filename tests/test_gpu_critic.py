"""Critic targets on the GPU (toget_critic_targets) against the oracle's
definition applied to the GPU's own returned trajectories: the same states
and controls enter both, so the float64 window sums agree to rounding."""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


@pytest.mark.parametrize("make,prec", [(W.pointmass, "fp64"), (W.planar3, "fp64"), (W.planar3, "mixed"),
                                       (W.arm7, "mixed")])
def test_critic_targets_match_the_definition(P, oracle_mod, make, prec):
    prob = make(seed=5)
    T_max = 60
    b = W.make_batch(prob, 24, seed=6, T=(5, T_max))
    h = P.tocreate_problem(prob.sys, prob.params, T_max)
    opts = P.to_default_opts(prec=P.TO_FP64 if prec == "fp64" else P.TO_MIXED, max_iter=6)
    bt = P.tosolve_batch(h, b.x0, b.T, opts=opts)
    r = P.toget_trajectories(bt)
    o = oracle_mod.Oracle.from_problem(prob)
    for K in (1, 7, T_max):
        V = P.toget_critic_targets(bt, K)
        for i in range(24):
            T = int(b.T[i])
            ref = o.critic_targets(r["X"][i, :T + 1], r["U"][i, :T], K)
            np.testing.assert_allclose(V[i, :T + 1], ref, rtol=1e-12, atol=0)
            assert np.all(V[i, T + 1:] == 0)
        if K == T_max:
            # the whole-horizon window is the solve's final cost (in mixed mode
            # the solver's own J comes from float32 cost evaluations: a small
            # terminal distance |ee - target| loses digits to cancellation)
            np.testing.assert_allclose(V[:, 0], r["J"], rtol=1e-12 if prec == "fp64" else 1e-5)


def test_critic_targets_reject_bad_window(P):
    prob = W.pointmass(seed=1)
    h = P.tocreate_problem(prob.sys, prob.params, 50)
    b = W.make_batch(prob, 4, seed=1)
    bt = P.tosolve_batch(h, b.x0, b.T, opts=P.to_default_opts(prec=P.TO_FP64, max_iter=3))
    with pytest.raises(P.ToError) as e:
        P.toget_critic_targets(bt, 0)
    assert e.value.code == P.TO_ERR_ARG
