"""Serving: continuous batching over the persistent kernel.

* a request's result is the same alone and in a mix of many concurrent
  requests of three systems and mixed horizons (the per-instance computation
  does not depend on co-residents);
* it equals the batch API's result for the same instance;
* admission is gated by the HBM budget (a one-seat server refuses a second
  request until the first is polled).
"""
import time

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


def _wait(server, rid, problem=None, want_traj=False, timeout=120.0):
    t0 = time.time()
    while True:
        r = server.poll(rid, problem, want_traj)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(1e-4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_alone_equals_in_the_mix(P, prec):
    probs = [W.pointmass(seed=1), W.planar3(seed=1), W.arm7(seed=1)]
    T_max = 120
    handles = [P.tocreate_problem(p.sys, p.params, T_max) for p in probs]
    opts = P.to_default_opts(prec=P.TO_FP64 if prec == "fp64" else P.TO_MIXED, max_iter=15)
    server = P.Server(handles, opts, hbm_budget_bytes=1 << 30)
    x_probe = W.make_batch(probs[1], 1, seed=9, T=90).x0[0]
    alone = _wait(server, server.submit(1, x_probe, 90), 1, want_traj=True)
    rng = np.random.default_rng(0)
    ids = []
    probe_id = None
    for k in range(240):
        pi = int(rng.integers(0, 3))
        Tk = int(rng.integers(50, T_max + 1))
        x0 = W.make_batch(probs[pi], 1, seed=int(rng.integers(1 << 30)), T=Tk).x0[0]
        ids.append((server.submit(pi, x0, Tk), pi))
        if k == 120:
            probe_id = server.submit(1, x_probe, 90)       # the probe joins mid-stream
    mixed = _wait(server, probe_id, 1, want_traj=True)
    for rid, pi in ids:
        r = _wait(server, rid)
        assert r["status"] & 15 in (1, 2, 3)
    assert mixed["iters"] == alone["iters"] and mixed["status"] == alone["status"]
    assert mixed["J"] == alone["J"]
    np.testing.assert_array_equal(mixed["X"], alone["X"])
    np.testing.assert_array_equal(mixed["U"], alone["U"])
    st = server.stats()
    assert st["busy"] == 0 and st["completed"] == 242
    server.close()


def test_served_result_equals_batch_api(P):
    prob = W.planar3(seed=3)
    T_max = 100
    h = P.tocreate_problem(prob.sys, prob.params, T_max)
    opts = P.to_default_opts(prec=P.TO_FP64, max_iter=12)
    b = W.make_batch(prob, 4, seed=4, T=(40, 100))
    bt = P.tosolve_batch(h, b.x0, b.T, opts=P.to_default_opts(prec=P.TO_FP64, max_iter=12))
    ref = P.toget_trajectories(bt)
    server = P.Server([h], opts, hbm_budget_bytes=256 << 20)
    for i in range(4):
        r = _wait(server, server.submit(0, b.x0[i], int(b.T[i])), 0, want_traj=True)
        assert r["iters"] == ref["iters"][i]
        assert abs(r["J"] - ref["J"][i]) <= 1e-12 * abs(ref["J"][i])
        np.testing.assert_allclose(r["X"], ref["X"][i], rtol=0, atol=1e-12 * np.abs(ref["X"][i]).max())
    server.close()


def test_admission_by_hbm_budget(P):
    prob = W.pointmass(seed=2)
    h = P.tocreate_problem(prob.sys, prob.params, 50)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=10)
    # a budget that holds exactly one request workspace
    # knot record x, u, x_lo padded to 12 floats; gain record 10 -> 12 floats
    per_seat = 51 * (17 * 12 + 12) * 4 + 11 * 12 + 64
    server = P.Server([h], opts, hbm_budget_bytes=per_seat + 100)
    assert server.stats()["seats"] == 1
    x = W.make_batch(prob, 2, seed=1).x0
    first = server.submit(0, x[0], 50)
    with pytest.raises(P.ToError) as e:
        server.submit(0, x[1], 50)
    assert e.value.code == P.TO_ERR_BUDGET
    _wait(server, first)
    second = server.submit(0, x[1], 50)
    assert _wait(server, second)["status"] & 15 in (1, 2, 3)
    server.close()


def test_requests_across_closed_launches(P):
    """A launch with nothing to solve closes after about a millisecond; later
    requests start a successor.  Bursts after idle gaps are all served, and
    the same request gives the same result in every burst."""
    prob = W.pointmass(seed=5)
    h = P.tocreate_problem(prob.sys, prob.params, 80)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=10)
    server = P.Server([h], opts, hbm_budget_bytes=256 << 20)
    b = W.make_batch(prob, 16, seed=6, T=(20, 80))
    first = None
    for burst in range(4):
        time.sleep(0.02)          # well past the idle window: the previous launch has closed
        ids = [server.submit(0, b.x0[i], int(b.T[i])) for i in range(16)]
        res = [_wait(server, r, timeout=60.0) for r in ids]
        Js = np.array([r["J"] for r in res])
        if first is None:
            first = Js
        np.testing.assert_array_equal(Js, first)
    assert server.stats()["completed"] == 64
    server.close()


def test_replay_trace_of_three_systems(P):
    """toserve_replay drives a Poisson trace in real time; every request
    finishes with a valid status and a latency no shorter than zero."""
    systems = (W.POINTMASS, W.PLANAR3, W.ARM7)
    probs = [W.make_problem(s, 0) for s in systems]
    handles = [P.tocreate_problem(p.sys, p.params, 120) for p in probs]
    server = P.Server(handles, P.to_default_opts(prec=P.TO_MIXED, max_iter=10), hbm_budget_bytes=1 << 30)
    trace = W.serving_stream(2e3, 0.1, seed=3, systems=systems, T_range=(20, 120))
    t_arr = np.array([t for t, _, _, _ in trace])
    pidx = np.array([systems.index(s) for _, s, _, _ in trace], np.int32)
    Ts = np.array([T for _, _, T, _ in trace], np.int32)
    x0 = np.zeros((len(trace), 14))
    for i, (_, _, _, x) in enumerate(trace):
        x0[i, :x.size] = x
    lat, J, st = server.replay(t_arr, pidx, Ts, x0, timeout_s=120.0)
    assert len(trace) > 100
    assert np.all(np.isin(st & 15, [1, 2, 3]))
    assert np.all(lat >= 0) and np.all(np.isfinite(J))
    server.close()
