"""Staging depth (to_solver_opts.stage_depth): how many knots ahead a group
fetches the records it reads next.  The depth moves loads, not arithmetic:
a solve at depth 2 takes the same iterations, statuses and step sizes as
the solve at depth 1, at every group size that offers it, in both
precisions, with ragged horizons down to T = 1 (a knot with no record D
knots away), with the V_x pass and with the Levenberg-Marquardt variant.
Values agree to the rounding of the compiler's multiply-add fusion, which
may differ between two kernel instantiations; the planar arm's chaotic
dynamics amplify it with the iterations (measured on this batch, FP64 after
12 iterations: costs within 3.5e-10 relative, trajectories within 5e-8), so
the comparison stops after 4 iterations.  The autotuner
times both depths, and an invalid depth is refused before any launch.
"""
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


def _solve(P, h, x0, T, opts, want_vx=False):
    bt = P.tosolve_batch(h, x0, T, opts=opts)
    r = P.toget_trajectories(bt, Vx=want_vx, K=want_vx)
    r["alpha"] = P.toget_history(bt)[0]          # the accepted step index of every iteration
    return r


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("G", [4, 8, 16, 32])
def test_depth_two_equals_depth_one(P, prec, G):
    prob = W.planar3(seed=21)
    T_max = 70
    b = W.make_batch(prob, 150, seed=22, T=(1, T_max))
    b.T[:4] = [1, 2, 3, T_max]          # the ring's edge cases: fewer knots than its depth
    h = P.tocreate_problem(prob.sys, prob.params, T_max)
    pr = P.TO_FP64 if prec == "fp64" else P.TO_MIXED
    # the planar arm is chaotic: a rounding-level difference grows with the
    # iterations (FP64, 12 iterations: trajectories apart by 5e-8 relative
    # at the end of one instance's horizon), so the comparison runs 4
    it = 4
    out = {}
    for D in (1, 2):
        opts = P.to_default_opts(prec=pr, max_iter=it, group_lanes=G, groups_per_block=64 // G, stage_depth=D)
        out[D] = _solve(P, h, b.x0, b.T, opts)
    _agree(out[2], out[1], prec)
    assert np.isfinite(out[1]["J"]).all()


def _agree(r, ref, prec):
    """Same iterations, statuses and accepted step sizes; values to rounding."""
    for k in ("iters", "status", "alpha"):
        if k in ref:
            np.testing.assert_array_equal(r[k], ref[k], err_msg=k)
    rtol = 1e-9 if prec == "fp64" else 1e-5
    np.testing.assert_allclose(r["J"], ref["J"], rtol=rtol, atol=0)
    for k in ("X", "U", "Vx", "K"):
        if ref.get(k) is not None:
            scale = np.abs(ref[k]).max()
            np.testing.assert_allclose(r[k], ref[k], rtol=0, atol=(1e-8 if prec == "fp64" else 1e-4) * scale,
                                       err_msg=k)


def test_depth_two_value_gradient_and_lm(P):
    """The V_x pass (one more backward pass) and the Levenberg-Marquardt
    variant (backward passes redone with a larger mu) at depth 2."""
    prob = W.planar3(seed=23)
    T_max = 40
    b = W.make_batch(prob, 64, seed=24, T=(2, T_max))
    h = P.tocreate_problem(prob.sys, prob.params, T_max)
    for extra in (dict(want_vx=1), dict(reg=P.TO_REG_LM)):
        out = {}
        for D in (1, 2):
            opts = P.to_default_opts(prec=P.TO_FP64, max_iter=4, group_lanes=8, groups_per_block=8, stage_depth=D,
                                     **extra)
            out[D] = _solve(P, h, b.x0, b.T, opts, want_vx=bool(extra.get("want_vx")))
        _agree(out[2], out[1], "fp64")


def test_totune_times_both_depths(P):
    prob = W.planar3(seed=25)
    b = W.make_batch(prob, 1024, seed=26, T=(50, 120))
    h = P.tocreate_problem(prob.sys, prob.params, 120)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=2)
    rows = P.totune(h, b.x0, b.T, opts)
    depths = {(r["group_lanes"], r["stage_depth"]) for r in rows}
    for G in (4, 8, 16, 32):
        assert (G, 1) in depths and (G, 2) in depths, G
    assert (1, 2) not in depths                 # a single lane stages one knot ahead only
    best = min(rows, key=lambda r: r["ms"])
    assert (opts.group_lanes, opts.groups_per_block, opts.stage_depth) == \
        (best["group_lanes"], best["groups_per_block"], best["stage_depth"])
    # a solve that leaves the shape unset runs the tuned one, depth included
    o0 = P.to_default_opts(prec=P.TO_MIXED, max_iter=2)
    r0 = _solve(P, h, b.x0[:128], b.T[:128], o0)
    r1 = _solve(P, h, b.x0[:128], b.T[:128], opts)
    np.testing.assert_array_equal(r0["J"], r1["J"])


def test_depth_not_offered_is_refused(P):
    prob = W.planar3(seed=27)
    b = W.make_batch(prob, 8, seed=28, T=(5, 10))
    h = P.tocreate_problem(prob.sys, prob.params, 10)
    for kw in (dict(stage_depth=3), dict(stage_depth=-1), dict(stage_depth=2, group_lanes=1, groups_per_block=64)):
        with pytest.raises(P.ToError) as e:
            P.tosolve_batch(h, b.x0, b.T, opts=P.to_default_opts(**kw))
        assert e.value.code == P.TO_ERR_ARG, kw
    pm = W.pointmass(seed=29)
    hp = P.tocreate_problem(pm.sys, pm.params, 10)
    bp = W.make_batch(pm, 8, seed=30, T=(5, 10))
    with pytest.raises(P.ToError) as e:
        P.tosolve_batch(hp, bp.x0, bp.T, opts=P.to_default_opts(stage_depth=2))
    assert e.value.code == P.TO_ERR_ARG
