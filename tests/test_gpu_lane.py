"""Single-lane groups (group_lanes = 1: one thread per instance, every
per-knot matrix in registers) against the FP64 oracle, through the C ABI.

The same parity bars as the lane-group kernels: the oracle's accepted step
sequence replayed (1e-10 relative in FP64; 1e-4 on trajectories and 1e-6 on
converged final costs in mixed mode, on well-conditioned instances), unforced
solves that take the oracle's own steps (the one-step-at-a-time line search
accepts the same smallest j), the Levenberg-Marquardt variant, V_x and the
gains of the returned iterate, serving, and agreement with the lane-group
kernel."""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W
from test_gpu_parity import FP64_TOL, _check, _check_consistency, _replay, _sensitivity

pytestmark = pytest.mark.gpu

LANE = dict(group_lanes=1, groups_per_block=64)


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


def _prec(P, prec):
    return P.TO_FP64 if prec == "fp64" else P.TO_MIXED


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pointmass_replay_lane(P, oracle_mod, prec):
    prob = W.pointmass(seed=0)
    b = W.make_batch(prob, 64, seed=0)
    o = oracle_mod.Oracle.from_problem(prob)
    ro = o.solve(b.x0, b.T, max_iter=100, tol=1e-8, n_alpha=16)
    kappa = _sensitivity(o, b, ro, 100)
    rg = _replay(P, prob, b, ro, _prec(P, prec), 100, **LANE)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.mean() >= 0.9
    _check_consistency(o, b, rg, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("T,iters,B", [((20, 40), 5, 24), ((20, 120), 20, 24), ((1, 9), 12, 70)])
def test_planar3_replay_lane(P, oracle_mod, prec, T, iters, B):
    # the lane-group suite's instances; 70 short ones: two full warps and a
    # ragged third, horizons down to 1
    prob = W.planar3(seed=1)
    b = W.make_batch(prob, B, seed=2, T=T)
    o = oracle_mod.Oracle.from_problem(prob)
    ro = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8)
    kappa = _sensitivity(o, b, ro, iters)
    rg = _replay(P, prob, b, ro, _prec(P, prec), iters, T_max=128, **LANE)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.mean() >= (0.4 if prec == "fp64" else 0.2)
    _check_consistency(o, b, rg, prec, min_checked=b.x0.shape[0] // 4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dubins_replay_lane(P, oracle_mod, prec):
    prob = W.dubins(seed=2)
    b = W.make_batch(prob, 48, seed=3, T=(30, 100))
    o = oracle_mod.Oracle.from_problem(prob)
    iters = 30
    ro = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8)
    kappa = _sensitivity(o, b, ro, iters)
    rg = _replay(P, prob, b, ro, _prec(P, prec), iters, T_max=100, **LANE)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.mean() >= 0.25
    _check_consistency(o, b, rg, prec, min_checked=12)


@pytest.mark.parametrize("sysname", ["pointmass", "dubins"])
def test_unforced_lane_matches_oracle_choices(P, oracle_mod, sysname):
    # the line search of a single lane tries j = 0, 1, ... one at a time and
    # accepts the first strict decrease: the oracle's rule
    prob = W.pointmass(seed=3) if sysname == "pointmass" else W.dubins(seed=4)
    b = W.make_batch(prob, 64, seed=4, T=None if sysname == "pointmass" else 60)
    ro = oracle_mod.Oracle.from_problem(prob).solve(b.x0, b.T, max_iter=100, tol=1e-8, n_alpha=16)
    s = P.Solver(prob, T_max=int(b.T.max()), prec=P.TO_FP64, **LANE)
    rg = s.solve(b.x0, b.T, max_iter=100, tol=1e-8)
    same = np.all(rg["alpha_hist"] == ro["alpha_hist"], axis=1) & (rg["iters"] == ro["iters"])
    assert same.mean() >= (0.95 if sysname == "pointmass" else 0.8), same.mean()
    ej = np.abs(rg["J"] - ro["J"]) / np.abs(ro["J"])
    assert np.median(ej[same]) < FP64_TOL
    for i in range(b.x0.shape[0]):
        Jh = rg["J_hist"][i, :rg["iters"][i] + 1]
        assert np.all(np.diff(Jh) < 0)


def test_value_gradient_and_gains_lane(P, oracle_mod):
    prob = W.planar3(seed=4)
    b = W.make_batch(prob, 6, seed=5, T=(15, 40))
    o = oracle_mod.Oracle.from_problem(prob)
    ro = o.solve(b.x0, b.T, max_iter=6, want_vx=True, want_K=True)
    kappa = _sensitivity(o, b, ro, 6)
    s = P.Solver(prob, T_max=40, prec=P.TO_FP64, **LANE)
    rg = s.solve(b.x0, b.T, forced_alpha=ro["alpha_hist"], max_iter=6, want_vx=1, want=("X", "U", "Vx", "K"))
    for i in np.where(kappa < 1e-12)[0]:
        T = int(b.T[i])
        vo, vg = ro["Vx"][i, :T + 1], rg["Vx"][i, :T + 1]
        assert np.abs(vg - vo).max() < 1e-9 * np.abs(vo).max()
        ko, kg = ro["K"][i, :T], rg["K"][i, :T]
        assert np.abs(kg - ko).max() < 1e-8 * np.abs(ko).max()
    assert (kappa < 1e-12).sum() >= 3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_planar3_lm_replay_lane(P, oracle_mod, prec):
    from test_gpu_lm import _sensitivity_lm
    prob = W.planar3(seed=1)
    b = W.make_batch(prob, 24, seed=2, T=(20, 40))
    o = oracle_mod.Oracle.from_problem(prob)
    iters = 8
    ro = o.solve(b.x0, b.T, max_iter=iters, tol=1e-8, n_alpha=16, reg="lm")
    kappa = _sensitivity_lm(o, b, ro, iters)
    s = P.Solver(prob, T_max=40, prec=_prec(P, prec), reg=P.TO_REG_LM, **LANE)
    rg = s.solve(b.x0, b.T, forced_alpha=ro["alpha_hist"], max_iter=iters)
    well = _check(ro, rg, kappa, prec, b.T)
    assert well.sum() >= 4


def test_lane_equals_lane_groups(P):
    # the point mass is well conditioned: the two kernels differ only by the
    # compiler's multiply-add fusion
    prob = W.pointmass(seed=4)
    b = W.make_batch(prob, 200, seed=5, T=(20, 80))
    out = []
    for kw in (dict(group_lanes=8, groups_per_block=8), LANE, dict(group_lanes=1, groups_per_block=256)):
        s = P.Solver(prob, T_max=80, prec=P.TO_FP64, **kw)
        out.append(s.solve(b.x0, b.T, max_iter=6))
    for r in out[1:]:
        np.testing.assert_array_equal(r["iters"], out[0]["iters"])
        np.testing.assert_array_equal(r["alpha_hist"], out[0]["alpha_hist"])
        np.testing.assert_allclose(r["J"], out[0]["J"], rtol=1e-11, atol=0)
        np.testing.assert_allclose(r["X"], out[0]["X"], rtol=0, atol=1e-11 * np.abs(out[0]["X"]).max())


def test_served_lane_result_equals_batch(P):
    prob = W.planar3(seed=6)
    b = W.make_batch(prob, 40, seed=7, T=(20, 60))
    h = P.tocreate_problem(prob.sys, prob.params, 60)
    opts = P.to_default_opts(prec=P.TO_FP64, max_iter=12, **LANE)
    bt = P.tosolve_batch(h, b.x0, b.T, opts=opts)
    ref = P.toget_trajectories(bt)
    server = P.Server([h], opts, hbm_budget_bytes=256 << 20)
    try:
        ids = [server.submit(0, b.x0[i], int(b.T[i])) for i in range(40)]
        got = {}
        import time
        t0 = time.time()
        while len(got) < 40 and time.time() - t0 < 120:
            for i, rid in enumerate(ids):
                if i not in got:
                    r = server.poll(rid)
                    if r is not None:
                        got[i] = r
            time.sleep(0.002)
        assert len(got) == 40
        for i in range(40):
            assert got[i]["iters"] == ref["iters"][i]
            assert abs(got[i]["J"] - ref["J"][i]) <= 1e-12 * abs(ref["J"][i])
    finally:
        server.close()


def test_autotuner_measures_single_lane_shapes(P):
    prob = W.planar3(seed=0)
    b = W.make_batch(prob, 1024, seed=0)
    h = P.tocreate_problem(prob.sys, prob.params, 400)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=3)
    rows = P.totune(h, b.x0, b.T, opts)
    shapes = {(r["group_lanes"], r["groups_per_block"]) for r in rows}
    assert {(1, 32), (1, 64), (1, 128), (1, 256)} <= shapes
    assert (8, 8) in shapes
    assert all(r["ms"] > 0 for r in rows)
