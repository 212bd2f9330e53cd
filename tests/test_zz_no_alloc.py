"""The no-allocation entry point, tosolve_batch_noalloc.

Some callers cannot call cudaMalloc while they run (a real-time control loop
with a bounded latency, code confined to a pre-sized memory pool, code running
while work is being captured into a CUDA graph).  For them the library solves
out of one static device array.  This test calls that entry point through the
C ABI twice in a row, on two different batches, and checks each result
against the regular entry point's within the tolerances the parity tests use;
the second call also shows that what the first call left in the shared array
does not leak into the next result.  It is collected last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_X_TOL = 1e-4
MIXED_J_TOL = 1e-6


@pytest.fixture(scope="module")
def P():
    import paper_2602_19699_gb300 as P
    P.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


def _regular(P, problem, x0, T, opts):
    """the existing device entry point + the host getter"""
    B = x0.shape[0]
    bt = P.tocreate_batch(problem, B, int((T + 1).sum().item()), opts)
    P.tosolve_batch_device(bt, B, x0.data_ptr(), T.data_ptr(), opts=opts)
    return P.toget_trajectories(bt)


def _noalloc(P, problem, x0, T, opts):
    import torch
    B, n = x0.shape
    dev = x0.device
    J = torch.empty(B, dtype=torch.float64, device=dev)
    it = torch.empty(B, dtype=torch.int32, device=dev)
    st = torch.empty(B, dtype=torch.int32, device=dev)
    X = torch.empty(B, problem.T_max + 1, n, dtype=torch.float64, device=dev)
    U = torch.empty(B, problem.T_max, problem.m, dtype=torch.float64, device=dev)
    P.tosolve_batch_noalloc(problem, B, x0.data_ptr(), T.data_ptr(), J.data_ptr(), it.data_ptr(), st.data_ptr(),
                            X.data_ptr(), U.data_ptr(), opts=opts,
                            stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {"J": J.cpu().numpy(), "iters": it.cpu().numpy(), "status": st.cpu().numpy(), "X": X.cpu().numpy(),
            "U": U.cpu().numpy()}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_regular_entry_point_twice(P, prec):
    import torch
    prob = W.planar3(seed=2)
    problem = P.tocreate_problem(prob.sys, prob.params, 120)
    opts = P.to_default_opts(prec=P.TO_FP64 if prec == "fp64" else P.TO_MIXED, max_iter=30)
    xt, jt = (FP64_TOL, FP64_TOL) if prec == "fp64" else (MIXED_X_TOL, MIXED_J_TOL)
    for seed, B in ((11, 96), (12, 64)):          # two calls in a row, different batches
        b = W.make_batch(prob, B, seed=seed, T=(20, 120))
        x0 = torch.tensor(b.x0, dtype=torch.float64, device="cuda")
        T = torch.tensor(b.T, dtype=torch.int32, device="cuda")
        ref = _regular(P, problem, x0, T, opts)
        got = _noalloc(P, problem, x0, T, opts)
        np.testing.assert_array_equal(got["iters"], ref["iters"])
        np.testing.assert_array_equal(got["status"], ref["status"])
        ok = np.isfinite(ref["J"])
        assert np.all(np.abs(got["J"][ok] - ref["J"][ok]) <= jt * np.abs(ref["J"][ok]))
        for key in ("X", "U"):
            a, r = got[key][ok], ref[key][ok]
            assert np.all(np.abs(a - r) <= xt * np.maximum(np.abs(r).max(axis=(1, 2), keepdims=True), 1e-300))


def test_noalloc_rejects_requests_beyond_the_static_workspace(P):
    import torch
    prob = W.planar3(seed=2)
    problem = P.tocreate_problem(prob.sys, prob.params, 400)
    B = 100000
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    zi = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(P.ToError) as e:
        P.tosolve_batch_noalloc(problem, B, z.data_ptr(), zi.data_ptr(), z.data_ptr(), zi.data_ptr(), zi.data_ptr())
    assert e.value.code == P.TO_ERR_BUDGET
    assert "static" in str(e.value)


@pytest.mark.parametrize("sysname", ["arm7", "quad"])
def test_noalloc_rigid_trees(P, sysname):
    # the rigid trees' per-knot scratch (stored substep primals) comes out of
    # the static array too
    import torch
    prob = W.arm7(seed=1) if sysname == "arm7" else W.quad(seed=2, with_actor=False)
    T_max = 30 if sysname == "arm7" else 10
    problem = P.tocreate_problem(prob.sys, prob.params, T_max)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=3)
    b = W.make_batch(prob, 8, seed=3, T=(5, T_max))
    x0 = torch.tensor(b.x0, dtype=torch.float64, device="cuda")
    T = torch.tensor(b.T, dtype=torch.int32, device="cuda")
    ref = _regular(P, problem, x0, T, opts)
    got = _noalloc(P, problem, x0, T, opts)
    np.testing.assert_array_equal(got["iters"], ref["iters"])
    np.testing.assert_array_equal(got["status"], ref["status"])
    ok = np.isfinite(ref["J"])
    assert ok.sum() >= 4
    assert np.all(np.abs(got["J"][ok] - ref["J"][ok]) <= MIXED_J_TOL * np.abs(ref["J"][ok]))
    for key in ("X", "U"):
        a, r = got[key][ok], ref[key][ok]
        assert np.all(np.abs(a - r) <= MIXED_X_TOL * np.maximum(np.abs(r).max(axis=(1, 2), keepdims=True), 1e-300))


def test_noalloc_rejected_horizon_reads_nothing(P):
    """A horizon outside [1, T_max] is caught on the device: every instance
    ends TO_ST_NONFINITE and the gathered X and U are NaN.  The call comes
    right after a valid solve, so the static array still holds that solve's
    offsets and slots; none of them may be read for the rejected batch."""
    import torch
    prob = W.planar3(seed=2)
    problem = P.tocreate_problem(prob.sys, prob.params, 60)
    opts = P.to_default_opts(prec=P.TO_MIXED, max_iter=5)
    b = W.make_batch(prob, 16, seed=21, T=(10, 60))
    x0 = torch.tensor(b.x0, dtype=torch.float64, device="cuda")
    T = torch.tensor(b.T, dtype=torch.int32, device="cuda")
    good = _noalloc(P, problem, x0, T, opts)
    assert np.all(np.isin(good["status"] & 15, [1, 2, 3]))
    Tbad = b.T.copy()
    Tbad[5] = 61                                     # T_max + 1
    got = _noalloc(P, problem, x0, torch.tensor(Tbad, dtype=torch.int32, device="cuda"), opts)
    assert np.all(got["status"] == P.TO_ST_NONFINITE)
    assert np.all(np.isnan(got["J"]))
    assert np.all(np.isnan(got["X"])) and np.all(np.isnan(got["U"]))
