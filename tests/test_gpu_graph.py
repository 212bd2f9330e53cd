"""CUDA-graph solves of a multi-system batch and the launch-shape autotuner.

* a captured graph of three systems (point mass, planar arm, 7-DoF arm; each
  its own branch and persistent kernel) gives, per member, the same results
  as that member solved alone with tosolve_batch, and new inputs written into
  the staging between replays (other initial states, other horizons) are
  picked up;
* the launch shape changes the schedule, not the arithmetic: solves at every
  supported shape agree (to the rounding of the compiler's multiply-add
  fusion, which may differ between kernel instantiations);
* totune measures every valid shape, returns the fastest, and later solves
  with an unset shape use it.
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


def _alone(P, handle, x0, T, opts):
    bt = P.tosolve_batch(handle, x0, T, opts=opts)
    return P.toget_trajectories(bt)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_members_equal_separate_solves(P, prec):
    T_max = 120
    probs = [W.pointmass(seed=1), W.planar3(seed=2), W.arm7(seed=3)]
    Bs = [96, 160, 40]
    handles = [P.tocreate_problem(p.sys, p.params, T_max) for p in probs]
    opts = P.to_default_opts(prec=P.TO_FP64 if prec == "fp64" else P.TO_MIXED, max_iter=8)
    batches = [P.tocreate_batch(h, B, B * (T_max + 1), opts) for h, B in zip(handles, Bs)]
    g = P.Graph(batches, Bs, opts=opts, shares=[1.0, 2.0, 2.0])
    assert g.launch_count() == 9
    for rnd in range(2):
        data = []
        for i, (p, B) in enumerate(zip(probs, Bs)):
            b = W.make_batch(p, B, seed=10 * rnd + i, T=(30, T_max) if rnd == 0 else (5, 60))
            x0s, Ts = g.inputs(i)
            x0s[:] = b.x0
            Ts[:] = b.T
            data.append(b)
        g.launch()
        g.sync()
        for i, (h, b) in enumerate(zip(handles, data)):
            out = g.outputs(i)
            ref = _alone(P, h, b.x0, b.T, opts)
            np.testing.assert_array_equal(out["iters"], ref["iters"])
            np.testing.assert_array_equal(out["status"], ref["status"])
            np.testing.assert_array_equal(out["J"], ref["J"])
            np.testing.assert_array_equal(out["X"], ref["X"])
            np.testing.assert_array_equal(out["U"], ref["U"])
    g.close()


def test_launch_shape_does_not_change_results(P):
    # the point mass: a well-conditioned system, so the fusion rounding stays
    # at its own size (the planar arm is chaotic and amplifies it)
    prob = W.pointmass(seed=4)
    b = W.make_batch(prob, 200, seed=5, T=(20, 80))
    h = P.tocreate_problem(prob.sys, prob.params, 80)
    ref = None
    for G, gpb in [(8, 4), (8, 8), (16, 2), (16, 8), (32, 1), (32, 4)]:
        opts = P.to_default_opts(prec=P.TO_FP64, max_iter=6, group_lanes=G, groups_per_block=gpb)
        r = _alone(P, h, b.x0, b.T, opts)
        if ref is None:
            ref = r
            continue
        # each shape is its own kernel instantiation: the compiler may fuse
        # a different multiply-add pair, so equal up to that rounding
        np.testing.assert_array_equal(r["iters"], ref["iters"])
        np.testing.assert_allclose(r["J"], ref["J"], rtol=1e-11, atol=0)
        np.testing.assert_allclose(r["X"], ref["X"], rtol=0, atol=1e-11 * np.abs(ref["X"]).max())


def test_totune_picks_the_fastest_and_caches_it(P):
    prob = W.planar3(seed=6)
    b = W.make_batch(prob, 2048, seed=7, T=(50, 150))
    h = P.tocreate_problem(prob.sys, prob.params, 150)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=3)
    rows = P.totune(h, b.x0, b.T, opts)
    assert len(rows) >= 6                      # 3 group sizes x several CTA shapes
    best = min(rows, key=lambda r: r["ms"])
    assert (opts.group_lanes, opts.groups_per_block) == (best["group_lanes"], best["groups_per_block"])
    for r in rows:
        assert r["ms"] > 0 and r["ctas_per_sm"] >= 1
        assert r["group_lanes"] * r["groups_per_block"] <= 256
    # an unset shape now means the tuned one; the results equal an explicit solve at that shape
    o0 = P.to_default_opts(prec=P.TO_MIXED, max_iter=3)
    bt = P.tosolve_batch(h, b.x0[:256], b.T[:256], opts=o0)
    r0 = P.toget_trajectories(bt, X=False, U=False)
    r1 = _alone(P, h, b.x0[:256], b.T[:256], opts)
    np.testing.assert_array_equal(r0["J"], r1["J"])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fused_launch_equals_separate_solves(P, prec):
    """tosolve_systems: the 7-DoF arm, the planar arm and the point mass in one
    persistent launch give each system's own results (the fused kernel is its
    own instantiation: equal up to the compiler's multiply-add fusion, as for
    launch shapes)."""
    import torch
    T_max = 80
    probs = [W.pointmass(seed=1), W.planar3(seed=2), W.arm7(seed=3)]
    Bs = [300, 500, 120]
    opts = P.to_default_opts(prec=P.TO_FP64 if prec == "fp64" else P.TO_MIXED, max_iter=4)
    handles = [P.tocreate_problem(p.sys, p.params, T_max) for p in probs]
    data = [W.make_batch(p, B, seed=20 + i, T=(10, T_max)) for i, (p, B) in enumerate(zip(probs, Bs))]
    d_x0 = [torch.tensor(b.x0, dtype=torch.float64, device="cuda") for b in data]
    d_T = [torch.tensor(b.T, dtype=torch.int32, device="cuda") for b in data]
    fused = [P.tocreate_batch(h, B, B * (T_max + 1), opts) for h, B in zip(handles, Bs)]
    P.tosolve_systems(fused, Bs, [x.data_ptr() for x in d_x0], [t.data_ptr() for t in d_T], opts=opts)
    torch.cuda.synchronize()
    assert P.tolast_launch_count(fused[0]) == 4          # three horizon sorts and one solver launch
    for i, (h, b) in enumerate(zip(handles, data)):
        got = P.toget_trajectories(fused[i])
        ref = _alone(P, h, b.x0, b.T, opts)
        same = got["iters"] == ref["iters"]
        if prec == "fp64":
            assert same.all()
            rtol = 1e-9 if probs[i].sys == W.PLANAR3 else 1e-11
            np.testing.assert_allclose(got["J"], ref["J"], rtol=rtol, atol=0)
        else:
            # float32 rounding differences may flip a near-tie step choice
            assert same.mean() >= 0.95
            np.testing.assert_allclose(got["J"][same], ref["J"][same], rtol=1e-4, atol=0)
        np.testing.assert_array_equal(got["status"][same] & 15, ref["status"][same] & 15)


def test_totune_persisted_choice(P, tmp_path, monkeypatch):
    """With TO_TUNE_CACHE set, the tuned shape is written to the file and a
    later call with the same workload reads it back without timing."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TO_TUNE_CACHE", str(cache))
    prob = W.pointmass(seed=8)
    b = W.make_batch(prob, 1024, seed=9, T=(20, 50))
    h = P.tocreate_problem(prob.sys, prob.params, 50)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=3)
    rows = P.totune(h, b.x0, b.T, opts)
    assert len(rows) >= 4
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:3] == [str(opts.group_lanes), str(opts.groups_per_block)]
    assert lines[0].split()[4] == str(opts.stage_depth) == "1"     # the point mass stages one knot ahead
    # a new problem handle, the same workload: the stored shape, no timing
    h2 = P.tocreate_problem(prob.sys, prob.params, 50)
    opts2 = P.to_default_opts(prec=P.TO_MIXED, max_iter=3)
    rows2 = P.totune(h2, b.x0, b.T, opts2)
    assert len(rows2) == 1
    assert (opts2.group_lanes, opts2.groups_per_block) == (opts.group_lanes, opts.groups_per_block)
    assert len(cache.read_text().splitlines()) == 1
    # another precision is another key
    opts3 = P.to_default_opts(prec=P.TO_FP64, max_iter=3)
    assert len(P.totune(h2, b.x0, b.T, opts3)) >= 4
    assert len(cache.read_text().splitlines()) == 2
