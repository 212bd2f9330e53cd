"""The bounds-checked build (``TO_CHECKED=1``, include/to.h: toget_bounds_report).

A child process loads ``libto_checked.so``, in which every computed index of
the solver kernel is checked against the buffer it addresses, and runs small
solves down every path: both precisions, every group size of the planar arm
(1, 4, 8, 16, 32 lanes; staging depths 1 and 2), horizons from 1 to T_max in one batch, the
Levenberg-Marquardt variant, forced step sequences, a caller's warm start,
V_x and gains, the point mass, the Dubins car, the 7-DoF arm, the quadruped
(64 and 32 lanes), one launch over several systems, the no-allocation entry
point and the serving loop.  Every problem's report must show no violation,
and the results must match the release library's on the same inputs (equal
iteration counts and statuses; costs equal up to the compiler's
multiply-add fusion, which may differ between the two builds as it does
between kernel instantiations).

Nothing here plants a bad index on the GPU: the checks are exercised by the
solves' own indices only.
"""
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _pn(P, prec):
    return "fp64" if prec == P.TO_FP64 else "mixed"


def _cases(P, W):
    """(name, result dict) of every case; P is the loaded binding."""
    import torch
    out = {}
    reports = {}

    def keep(name, r, problem):
        out[name] = {k: np.asarray(r[k]).tolist() for k in ("J", "iters", "status") if k in r}
        if P.tobounds_checked():
            reports[name] = P.toget_bounds_report(problem, reset=True)

    # planar arm: ragged horizons 1 .. T_max, every group size, both precisions
    prob = W.planar3(seed=2)
    T_max = 60
    b = W.make_batch(prob, 48, seed=7, T=(1, T_max))
    b.T[0], b.T[1] = 1, T_max
    for prec in (P.TO_MIXED, P.TO_FP64):
        for G in (8, 1, 4, 16, 32):
            s = P.Solver(prob, T_max=T_max, prec=prec, group_lanes=G)
            r = s.solve(b.x0, b.T, max_iter=15)
            keep(f"planar_{_pn(P, prec)}_{G}", r, s.problem)
        for G in (4, 8, 16, 32):          # staging depth 2: records fetched two knots ahead
            s = P.Solver(prob, T_max=T_max, prec=prec, group_lanes=G, stage_depth=2)
            r = s.solve(b.x0, b.T, max_iter=15)
            keep(f"planar_{_pn(P, prec)}_{G}_d2", r, s.problem)
    # Levenberg-Marquardt, forced steps, a caller's warm start, V_x
    s = P.Solver(prob, T_max=T_max, prec=P.TO_MIXED, reg=P.TO_REG_LM)
    keep("planar_lm", s.solve(b.x0, b.T, max_iter=15), s.problem)
    s = P.Solver(prob, T_max=T_max, prec=P.TO_FP64)
    r0 = s.solve(b.x0, b.T, max_iter=6)
    keep("planar_fp64_forced", s.solve(b.x0, b.T, forced_alpha=r0["alpha_hist"], max_iter=6, want_vx=1,
                                  want=("X", "U", "Vx", "K")), s.problem)
    U0 = np.random.default_rng(3).normal(0, 0.1, (48, T_max, prob.m))
    keep("planar_fp64_uinit", s.solve(b.x0, b.T, U_init=U0, max_iter=6), s.problem)
    # the other systems
    for name, pr, Tm, B, it, kw in (("pointmass", W.pointmass(seed=1), 50, 40, 20, {}),
                                    ("dubins", W.dubins(seed=1), 50, 40, 20, {}),
                                    ("arm7", W.arm7(seed=1), 20, 8, 3, {}),
                                    ("quad64", W.quad(seed=2, with_actor=False), 4, 4, 1, {"group_lanes": 64}),
                                    ("quad32", W.quad(seed=2, with_actor=False), 4, 4, 1, {"group_lanes": 32})):
        bb = W.make_batch(pr, B, seed=5, T=(1, Tm) if Tm > 4 else Tm)
        for prec in (P.TO_MIXED, P.TO_FP64):
            s = P.Solver(pr, T_max=Tm, prec=prec, **kw)
            keep(f"{name}_{_pn(P, prec)}", s.solve(bb.x0, bb.T, max_iter=it), s.problem)
    # the quadruped's actor warm start
    pr = W.quad(seed=4, with_actor=True)
    bb = W.make_batch(pr, 3, seed=5, T=6)
    s = P.Solver(pr, T_max=6, prec=P.TO_MIXED)
    keep("quad_actor", s.solve(bb.x0, bb.T, max_iter=1), s.problem)
    # one launch over several systems
    probs = [W.pointmass(seed=1), W.planar3(seed=2), W.arm7(seed=3)]
    Bs = [30, 50, 12]
    Tm = 40
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=4)
    hs = [P.tocreate_problem(p.sys, p.params, Tm) for p in probs]
    data = [W.make_batch(p, B, seed=20 + i, T=(1, Tm)) for i, (p, B) in enumerate(zip(probs, Bs))]
    d_x0 = [torch.tensor(d.x0, dtype=torch.float64, device="cuda") for d in data]
    d_T = [torch.tensor(d.T, dtype=torch.int32, device="cuda") for d in data]
    bts = [P.tocreate_batch(h, B, B * (Tm + 1), opts) for h, B in zip(hs, Bs)]
    P.tosolve_systems(bts, Bs, [x.data_ptr() for x in d_x0], [t.data_ptr() for t in d_T], opts=opts)
    torch.cuda.synchronize()
    for i, (h, bt) in enumerate(zip(hs, bts)):
        keep(f"systems_{i}", P.toget_trajectories(bt, X=False, U=False), h)
    # the no-allocation entry point
    h = P.tocreate_problem(prob.sys, prob.params, T_max)
    x0 = torch.tensor(b.x0, dtype=torch.float64, device="cuda")
    Td = torch.tensor(b.T, dtype=torch.int32, device="cuda")
    J = torch.empty(48, dtype=torch.float64, device="cuda")
    it = torch.empty(48, dtype=torch.int32, device="cuda")
    st = torch.empty(48, dtype=torch.int32, device="cuda")
    P.tosolve_batch_noalloc(h, 48, x0.data_ptr(), Td.data_ptr(), J.data_ptr(), it.data_ptr(), st.data_ptr(),
                            opts=P.to_default_opts(prec=P.TO_MIXED, max_iter=10),
                            stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    keep("noalloc", {"J": J.cpu().numpy(), "iters": it.cpu().numpy(), "status": st.cpu().numpy()}, h)
    # serving: a few requests through the seats
    h = P.tocreate_problem(prob.sys, prob.params, T_max)
    server = P.Server([h], P.to_default_opts(prec=P.TO_FP64, max_iter=8), hbm_budget_bytes=64 << 20)
    res = {"J": [], "iters": [], "status": []}
    for i in range(4):
        rid = server.submit(0, b.x0[i], int(b.T[i]))
        t0 = time.time()
        while True:
            r = server.poll(rid, 0, False)
            if r is not None:
                break
            assert time.time() - t0 < 120.0, "request did not finish"
            time.sleep(1e-4)
        for k in res:
            res[k].append(r[k])
    server.close()
    keep("serve_fp64", res, h)
    return out, reports


def _child(path):
    """Run every case on the checked library and write results and reports."""
    import paper_2602_19699_gb300 as P
    from paper_2602_19699_gb300 import workload as W
    assert P.CHECKED
    P.build()
    assert P.tobounds_checked()
    out, reports = _cases(P, W)
    with open(path, "w") as f:
        json.dump({"results": out, "reports": reports}, f)


@pytest.mark.gpu
def test_checked_build_reports_no_violation_and_matches_release(tmp_path):
    import paper_2602_19699_gb300 as P
    from paper_2602_19699_gb300 import workload as W
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    assert not P.CHECKED
    P.build()
    assert not P.tobounds_checked()
    path = str(tmp_path / "checked.json")
    env = dict(os.environ, TO_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), path], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = json.load(open(path))
    reports = got["reports"]
    assert reports, "the checked build returned no report"
    bad = {k: v for k, v in reports.items() if v["violations"]}
    assert not bad, bad
    # the release library on the same inputs
    ref, rep = _cases(P, W)
    assert rep == {}
    with pytest.raises(P.ToError) as e:
        P.toget_bounds_report(P.tocreate_problem(W.PLANAR3, W.planar3(seed=2).params, 10))
    assert e.value.code == P.TO_ERR_UNSUPPORTED
    assert set(ref) == set(got["results"])
    for name, a in got["results"].items():
        b = ref[name]
        ia, ib = np.asarray(a["iters"]), np.asarray(b["iters"])
        same = ia == ib
        fp64 = "fp64" in name
        assert same.all() if fp64 else same.mean() >= 0.9, (name, ia, ib)
        np.testing.assert_array_equal(np.asarray(a["status"])[same] & 15, np.asarray(b["status"])[same] & 15)
        Ja, Jb = np.asarray(a["J"], float)[same], np.asarray(b["J"], float)[same]
        ok = np.isfinite(Jb)
        np.testing.assert_allclose(Ja[ok], Jb[ok], rtol=1e-9 if fp64 else 1e-4, atol=0, err_msg=name)


if __name__ == "__main__":
    _child(sys.argv[1])
