"""Python binding of libto.so, the GB300 batched iLQR library (include/to.h).

The functions keep the C names (``tocreate_problem``, ``tosolve_batch``,
``toget_trajectories`` ...) and only marshal arguments: every step of the
solve runs in the CUDA kernels of the shared library.  There is no CPU
fallback: calling into the library without a built ``libto.so`` or without a
CUDA device raises.

``Solver`` is a small convenience wrapper (one problem + one reusable batch).

With the environment variable ``TO_CHECKED=1`` the binding loads the
bounds-checked build ``_lib/libto_checked.so`` (``build(checked=True)``)
instead of the release library.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
CHECKED = os.environ.get("TO_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "_lib", "libto_checked.so" if CHECKED else "libto.so")

TO_SYS_POINTMASS2D, TO_SYS_PLANAR3, TO_SYS_ARM7, TO_SYS_QUAD18, TO_SYS_DUBINS = 1, 2, 3, 4, 5
TO_FP64, TO_MIXED = 0, 1
TO_OK, TO_ERR_ARG, TO_ERR_CUDA, TO_ERR_BUDGET, TO_ERR_TIMEOUT, TO_ERR_NOTREADY, TO_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
TO_ST_CONVERGED, TO_ST_MAX_ITER, TO_ST_LS_FAIL, TO_ST_NONFINITE, TO_ST_TIMEOUT, TO_ST_FLAG_REG = 1, 2, 3, 4, 5, 16
TO_REG_CLIP, TO_REG_LM = 0, 1


class ToError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libto error {code}: {msg}")
        self.code = code


class to_problem_desc(C.Structure):
    _fields_ = [("sys", C.c_int), ("n", C.c_int), ("m", C.c_int), ("T_max", C.c_int), ("dt", C.c_double),
                ("params", C.POINTER(C.c_double)), ("n_params", C.c_size_t),
                ("actor_w", C.POINTER(C.c_float)), ("n_actor_w", C.c_size_t), ("u_max", C.c_double)]


class to_solver_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("tol_rel", C.c_double), ("eps_clip", C.c_double), ("n_alpha", C.c_int),
                ("alpha_decay", C.c_double), ("prec", C.c_int), ("refine", C.c_int),
                ("forced_alpha", C.POINTER(C.c_int)), ("want_vx", C.c_int), ("hbm_budget_bytes", C.c_size_t),
                ("group_lanes", C.c_int), ("groups_per_block", C.c_int), ("profile_phases", C.c_int),
                ("reg", C.c_int), ("stage_depth", C.c_int)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False, checked: bool = CHECKED) -> str:
    from . import nvcc_build as _b
    return _b.build(force=force, checked=checked)


def lib():
    """The loaded libto.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); "
                                   f"run paper_2602_19699_gb300.build({'checked=True' if CHECKED else ''})")
            L = C.CDLL(LIB_PATH)
            vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
            L.tocreate_problem.argtypes = [C.POINTER(to_problem_desc), C.POINTER(vp)]
            L.todestroy_problem.argtypes = [vp]
            L.todestroy_problem.restype = None
            L.tocreate_batch.argtypes = [vp, i, ll, C.POINTER(to_solver_opts), C.POINTER(vp)]
            L.tofree_batch.argtypes = [vp]
            L.tofree_batch.restype = None
            L.tosolve_batch.argtypes = [vp, i, vp, vp, vp, C.POINTER(to_solver_opts), vp, C.POINTER(vp)]
            L.tosolve_batch_device.argtypes = [vp, i, vp, vp, vp, vp, C.POINTER(to_solver_opts), vp]
            L.toget_trajectories.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.toget_history.argtypes = [vp, vp, vp]
            L.toget_device_results.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
            L.tolast_launch_count.argtypes = [vp]
            L.toget_phase_cycles.argtypes = [vp, vp]
            L.tobounds_checked.argtypes = []
            L.toget_bounds_report.argtypes = [vp, vp, i]
            L.tosolve_batch_noalloc.argtypes = [vp, i, vp, vp, C.POINTER(to_solver_opts), vp, vp, vp, vp, vp, vp]
            L.tosolve_systems.argtypes = [vp, vp, vp, vp, i, C.POINTER(to_solver_opts), vp]
            L.toserver_create.argtypes = [vp, i, C.POINTER(to_solver_opts), C.c_size_t, C.POINTER(vp)]
            L.toserver_destroy.argtypes = [vp]
            L.toserver_destroy.restype = None
            L.tosubmit.argtypes = [vp, i, vp, i, C.POINTER(C.c_uint64)]
            L.topoll.argtypes = [vp, C.c_uint64, vp, vp, vp, vp, vp, vp]
            L.toserver_stats.argtypes = [vp, vp, vp, vp, vp]
            L.toserve_replay.argtypes = [vp, i, vp, vp, vp, vp, i, vp, vp, vp, d]
            L.toget_critic_targets.argtypes = [vp, i, vp]
            L.toranker_create.argtypes = [i, vp, C.c_size_t, C.POINTER(vp)]
            L.torank_candidates.argtypes = [vp, i, vp, i, vp, vp, vp]
            L.toranker_destroy.argtypes = [vp]
            L.toranker_destroy.restype = None
            L.totune.argtypes = [vp, i, vp, vp, C.POINTER(to_solver_opts), vp, i, vp]
            L.tograph_create.argtypes = [vp, vp, vp, i, C.POINTER(to_solver_opts), i, C.POINTER(vp)]
            L.tograph_staging.argtypes = [vp, i] + [C.POINTER(vp)] * 7
            L.tograph_launch.argtypes = [vp, vp]
            L.tograph_sync.argtypes = [vp]
            L.tograph_launch_count.argtypes = [vp]
            L.tograph_destroy.argtypes = [vp]
            L.tograph_destroy.restype = None
            L.tolast_error.restype = C.c_char_p
            L.to_default_opts.argtypes = [C.POINTER(to_solver_opts)]
            L.to_default_opts.restype = None
            _lib = L
    return _lib


def exported_symbols():
    return ["to_default_opts", "tocreate_problem", "todestroy_problem", "tocreate_batch", "tofree_batch",
            "tosolve_batch", "tosolve_batch_device", "toget_trajectories", "toget_history",
            "toget_device_results", "tolast_launch_count", "toget_phase_cycles", "tosolve_batch_noalloc",
            "tosolve_systems",
            "toserver_create", "toserver_destroy", "tosubmit", "topoll", "toserver_stats", "toserve_replay",
            "toget_critic_targets", "toranker_create", "torank_candidates", "toranker_destroy", "totune",
            "tograph_create", "tograph_staging", "tograph_launch", "tograph_sync", "tograph_launch_count",
            "tograph_destroy", "tolast_error", "tobounds_checked", "toget_bounds_report"]


class Ranker:
    """Biased-initial-condition ranking with the std-critic MLP (toranker_*)."""

    def __init__(self, n_in: int, weights):
        self.w = np.ascontiguousarray(weights, dtype=np.float32)
        self.handle = C.c_void_p()
        _check(lib().toranker_create(int(n_in), _ptr(self.w), self.w.size, C.byref(self.handle)))
        self.n_in = int(n_in)

    def rank(self, x, N: int, want_scores: bool = False, stream=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        Cn = x.shape[0]
        idx = np.empty(int(N), np.int32)
        sc = np.empty(Cn, np.float32) if want_scores else None
        _check(lib().torank_candidates(self.handle, Cn, _ptr(x), int(N), _ptr(idx), _ptr(sc) if sc is not None else None,
                                       stream))
        return (idx, sc) if want_scores else idx

    def close(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.toranker_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        self.close()


class to_tune_row(C.Structure):
    _fields_ = [("group_lanes", C.c_int), ("groups_per_block", C.c_int), ("grid", C.c_int),
                ("ctas_per_sm", C.c_int), ("ms", C.c_double), ("stage_depth", C.c_int)]


def totune(problem: "Problem", x0, T, opts: "to_solver_opts", max_rows: int = 64):
    """Time every valid launch shape on the calibration batch (x0, T); the
    fastest is written into ``opts`` and cached in the problem.  Returns the
    measured rows as dicts."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    rows = (to_tune_row * max_rows)()
    n = C.c_int()
    _check(lib().totune(problem.handle, int(T.size), _ptr(x0), _ptr(T), C.byref(opts), rows, max_rows, C.byref(n)))
    return [{"group_lanes": r.group_lanes, "groups_per_block": r.groups_per_block, "grid": r.grid,
             "ctas_per_sm": r.ctas_per_sm, "ms": r.ms, "stage_depth": r.stage_depth} for r in rows[:n.value]]


class Graph:
    """A captured multi-system solve (one member batch per problem).  Fill
    ``inputs(i)`` (pinned x0, T views), ``launch()``, ``sync()``, read
    ``outputs(i)`` (pinned views, valid until the next launch)."""

    def __init__(self, batches, B, opts: "to_solver_opts | None" = None, shares=None, want_traj: bool = True):
        self.batches = list(batches)
        self.B = [int(b) for b in B]
        hb = (C.c_void_p * len(self.batches))(*[b.handle.value for b in self.batches])
        Bs = (C.c_int * len(self.B))(*self.B)
        sh = None if shares is None else (C.c_double * len(shares))(*[float(x) for x in shares])
        self.handle = C.c_void_p()
        self.want_traj = bool(want_traj)
        _check(lib().tograph_create(hb, Bs, sh, len(self.batches), C.byref(opts) if opts else None,
                                    int(self.want_traj), C.byref(self.handle)))
        self._views = [self._member_views(i) for i in range(len(self.batches))]
        for bt, Bi in zip(self.batches, self.B):
            bt.B = Bi
            bt.max_iter = opts.max_iter if opts else 100

    def _member_views(self, i):
        ptrs = [C.c_void_p() for _ in range(7)]
        _check(lib().tograph_staging(self.handle, i, *[C.byref(p) for p in ptrs]))
        prob = self.batches[i].problem
        B = self.B[i]

        def view(p, shape, ctype, dtype):
            if not p.value:
                return None
            n = int(np.prod(shape))
            return np.ctypeslib.as_array(C.cast(p, C.POINTER(ctype)), shape=(n,)).view(dtype).reshape(shape)
        return {"x0": view(ptrs[0], (B, prob.n), C.c_double, np.float64),
                "T": view(ptrs[1], (B,), C.c_int, np.int32),
                "X": view(ptrs[2], (B, prob.T_max + 1, prob.n), C.c_double, np.float64),
                "U": view(ptrs[3], (B, prob.T_max, prob.m), C.c_double, np.float64),
                "J": view(ptrs[4], (B,), C.c_double, np.float64),
                "iters": view(ptrs[5], (B,), C.c_int, np.int32),
                "status": view(ptrs[6], (B,), C.c_int, np.int32)}

    def inputs(self, i):
        v = self._views[i]
        return v["x0"], v["T"]

    def outputs(self, i):
        v = self._views[i]
        return {k: v[k] for k in ("X", "U", "J", "iters", "status")}

    def launch(self, stream=None):
        _check(lib().tograph_launch(self.handle, stream))

    def sync(self):
        _check(lib().tograph_sync(self.handle))

    def launch_count(self) -> int:
        return lib().tograph_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.tograph_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        self.close()


class Server:
    """Continuous-batching server over several problems (see include/to.h)."""

    def __init__(self, problems, opts: to_solver_opts | None = None, hbm_budget_bytes: int = 0):
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        self.handle = C.c_void_p()
        _check(lib().toserver_create(arr, len(self.problems), C.byref(opts) if opts else None,
                                     int(hbm_budget_bytes), C.byref(self.handle)))

    def submit(self, problem: int, x0, T: int) -> int:
        x = np.ascontiguousarray(x0, dtype=np.float64)
        rid = C.c_uint64()
        _check(lib().tosubmit(self.handle, int(problem), _ptr(x), int(T), C.byref(rid)))
        return rid.value

    def poll(self, req_id: int, problem: int | None = None, want_traj: bool = False):
        """None while running; else dict(J, iters, status, latency_ms[, X, U])."""
        J, it, st, lat = C.c_double(), C.c_int(), C.c_int(), C.c_double()
        X = U = None
        if want_traj:
            p = self.problems[problem]
            X = np.empty((p.T_max + 1, p.n))
            U = np.empty((p.T_max, p.m))
        rc = lib().topoll(self.handle, C.c_uint64(req_id), _ptr(X), _ptr(U), C.byref(J), C.byref(it), C.byref(st),
                          C.byref(lat))
        if rc == TO_ERR_NOTREADY:
            return None
        _check(rc)
        out = {"J": J.value, "iters": it.value, "status": st.value, "latency_ms": lat.value}
        if want_traj:
            out["X"], out["U"] = X, U
        return out

    def stats(self):
        tot, busy, done, nbytes = C.c_int(), C.c_int(), C.c_longlong(), C.c_size_t()
        _check(lib().toserver_stats(self.handle, C.byref(tot), C.byref(busy), C.byref(done), C.byref(nbytes)))
        return {"seats": tot.value, "busy": busy.value, "completed": done.value, "hbm_bytes": nbytes.value}

    def replay(self, arrival_s, problem, T, x0, timeout_s: float = 600.0):
        """Real-time replay of a request trace; returns (latency_ms, J, status)."""
        arrival_s = np.ascontiguousarray(arrival_s, dtype=np.float64)
        problem = np.ascontiguousarray(problem, dtype=np.int32)
        T = np.ascontiguousarray(T, dtype=np.int32)
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        n = arrival_s.size
        lat, J, st = np.empty(n), np.empty(n), np.empty(n, np.int32)
        _check(lib().toserve_replay(self.handle, n, _ptr(arrival_s), _ptr(problem), _ptr(T), _ptr(x0), x0.shape[1],
                                    _ptr(lat), _ptr(J), _ptr(st), C.c_double(timeout_s)))
        return lat, J, st

    def close(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.toserver_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        self.close()


def tolast_error() -> str:
    return lib().tolast_error().decode()


def _check(rc):
    if rc != TO_OK:
        raise ToError(rc, tolast_error())


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def to_default_opts(**overrides) -> to_solver_opts:
    o = to_solver_opts()
    lib().to_default_opts(C.byref(o))
    for k, v in overrides.items():
        if k == "forced_alpha":
            raise ValueError("pass forced_alpha to tosolve_batch")
        setattr(o, k, v)
    return o


class Problem:
    """Handle of a created problem (keeps the host parameter copy alive)."""

    def __init__(self, handle, sys, n, m, T_max):
        self.handle, self.sys, self.n, self.m, self.T_max = handle, sys, n, m, T_max

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.todestroy_problem(self.handle)
            self.handle = None


class Batch:
    def __init__(self, handle, problem):
        self.handle, self.problem = handle, problem
        self.B = 0
        self.max_iter = 0
        self.want_vx = 0

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tofree_batch(self.handle)
            self.handle = None


def tocreate_problem(sys, params, T_max, actor_w=None, n=None, m=None, dt=None) -> Problem:
    from .workload import NM
    n0, m0 = NM.get(sys, (0, 0))
    p = np.ascontiguousarray(params, dtype=np.float64)
    d = to_problem_desc()
    d.sys = sys
    d.n = n0 if n is None else n
    d.m = m0 if m is None else m
    d.T_max = int(T_max)
    d.dt = float(p[0]) if dt is None else dt
    d.params = p.ctypes.data_as(C.POINTER(C.c_double))
    d.n_params = p.size
    aw = None
    if actor_w is not None:
        aw = np.ascontiguousarray(actor_w, dtype=np.float32)
        d.actor_w = aw.ctypes.data_as(C.POINTER(C.c_float))
        d.n_actor_w = aw.size
    d.u_max = float("inf")
    h = C.c_void_p()
    _check(lib().tocreate_problem(C.byref(d), C.byref(h)))
    return Problem(h, sys, d.n, d.m, d.T_max)


def tocreate_batch(problem: Problem, B_max: int, knots_max: int, opts: to_solver_opts | None = None) -> Batch:
    h = C.c_void_p()
    _check(lib().tocreate_batch(problem.handle, int(B_max), int(knots_max), C.byref(opts) if opts else None,
                                C.byref(h)))
    return Batch(h, problem)


def tosolve_batch(problem: Problem, x0, T, U_init=None, opts: to_solver_opts | None = None, stream=None,
                  batch: Batch | None = None, forced_alpha=None) -> Batch:
    """Solve with host inputs; returns the (possibly new) batch.  Asynchronous on ``stream``."""
    x0 = np.ascontiguousarray(np.atleast_2d(x0), dtype=np.float64)
    B = x0.shape[0]
    T = np.ascontiguousarray(np.broadcast_to(np.asarray(T), (B,)), dtype=np.int32)
    opts = opts if opts is not None else to_default_opts()
    fa = None
    if forced_alpha is not None:
        fa = np.ascontiguousarray(forced_alpha, dtype=np.int32)
        assert fa.shape == (B, opts.max_iter)
        opts.forced_alpha = fa.ctypes.data_as(C.POINTER(C.c_int))
    else:
        opts.forced_alpha = None
    U = None
    if U_init is not None:
        U = np.ascontiguousarray(U_init, dtype=np.float64)
        assert U.shape == (B, problem.T_max, problem.m)
    h = C.c_void_p(batch.handle.value if batch is not None else None)
    rc = lib().tosolve_batch(problem.handle, B, _ptr(x0), _ptr(T), _ptr(U), C.byref(opts),
                             C.c_void_p(stream) if stream else None, C.byref(h))
    opts.forced_alpha = None
    _check(rc)
    if batch is None:
        batch = Batch(h, problem)
    batch.B, batch.max_iter, batch.want_vx = B, opts.max_iter, opts.want_vx
    return batch


def tosolve_batch_device(batch: Batch, B: int, d_x0: int, d_T: int, d_U_init: int | None = None,
                         d_forced: int | None = None, opts: to_solver_opts | None = None, stream=None):
    """Solve with device-resident inputs (raw device pointers, e.g. torch ``data_ptr()``)."""
    opts = opts if opts is not None else to_default_opts()
    opts.forced_alpha = None
    _check(lib().tosolve_batch_device(batch.handle, int(B), C.c_void_p(d_x0), C.c_void_p(d_T),
                                      C.c_void_p(d_U_init) if d_U_init else None,
                                      C.c_void_p(d_forced) if d_forced else None, C.byref(opts),
                                      C.c_void_p(stream) if stream else None))
    batch.B, batch.max_iter, batch.want_vx = B, opts.max_iter, opts.want_vx


def tosolve_systems(batches, Bs, d_x0s, d_Ts, opts: to_solver_opts | None = None, stream=None):
    """Several systems (7-DoF arm, planar arm, point mass; one batch each) in
    one persistent launch, from device-resident inputs (raw device pointers)."""
    opts = opts if opts is not None else to_default_opts()
    opts.forced_alpha = None
    n = len(batches)
    hb = (C.c_void_p * n)(*[b.handle.value for b in batches])
    Bv = (C.c_int * n)(*[int(B) for B in Bs])
    xv = (C.c_void_p * n)(*[int(p) for p in d_x0s])
    tv = (C.c_void_p * n)(*[int(p) for p in d_Ts])
    _check(lib().tosolve_systems(hb, Bv, xv, tv, n, C.byref(opts), C.c_void_p(stream) if stream else None))
    for b, B in zip(batches, Bs):
        b.B, b.max_iter, b.want_vx = int(B), opts.max_iter, 0


def tosolve_batch_noalloc(problem: Problem, B: int, d_x0: int, d_T: int, d_J: int, d_iters: int, d_status: int,
                          d_X: int | None = None, d_U: int | None = None, opts: to_solver_opts | None = None,
                          stream=None):
    """Solve without allocating device memory: the library's static workspace
    is used and the caller's device buffers receive the results (raw device
    pointers).  The first call on a device must come before any stream capture;
    calls that overlap on the GPU race on the shared workspace."""
    opts = opts if opts is not None else to_default_opts()
    opts.forced_alpha = None
    vp = C.c_void_p
    _check(lib().tosolve_batch_noalloc(problem.handle, int(B), vp(d_x0), vp(d_T), C.byref(opts),
                                       vp(stream) if stream else None, vp(d_J), vp(d_iters), vp(d_status),
                                       vp(d_X) if d_X else None, vp(d_U) if d_U else None))


def toget_trajectories(batch: Batch, X=True, U=True, Vx=False, K=False) -> dict:
    p = batch.problem
    B = batch.B
    out = {
        "J": np.empty(B), "iters": np.empty(B, np.int32), "status": np.empty(B, np.int32),
        "X": np.empty((B, p.T_max + 1, p.n)) if X else None,
        "U": np.empty((B, p.T_max, p.m)) if U else None,
        "Vx": np.empty((B, p.T_max + 1, p.n)) if Vx else None,
        "K": np.empty((B, p.T_max, p.m, p.n)) if K else None,
    }
    _check(lib().toget_trajectories(batch.handle, _ptr(out["X"]), _ptr(out["U"]), _ptr(out["J"]),
                                    _ptr(out["iters"]), _ptr(out["status"]), _ptr(out["Vx"]), _ptr(out["K"])))
    return out


def toget_critic_targets(batch: Batch, K: int) -> np.ndarray:
    """Partial K-step cost-to-go of every knot of the last solve, B x (T_max+1)."""
    out = np.empty((batch.B, batch.problem.T_max + 1))
    _check(lib().toget_critic_targets(batch.handle, int(K), _ptr(out)))
    return out


def toget_history(batch: Batch) -> tuple[np.ndarray, np.ndarray]:
    B, mi = batch.B, batch.max_iter
    a = np.empty((B, max(mi, 1)), np.int32)
    j = np.empty((B, mi + 1))
    _check(lib().toget_history(batch.handle, _ptr(a), _ptr(j)))
    return a[:, :mi], j


def toget_device_results(batch: Batch) -> tuple[int, int, int]:
    J, it, st = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(lib().toget_device_results(batch.handle, C.byref(J), C.byref(it), C.byref(st)))
    return J.value, it.value, st.value


PHASES = ("bookkeeping", "bwd_derivs", "bwd_products", "bwd_chol_gains", "bwd_update", "line_search", "commit")


def toget_phase_cycles(batch: Batch) -> dict:
    out = np.zeros(8, np.uint64)
    _check(lib().toget_phase_cycles(batch.handle, _ptr(out)))
    d = {k: int(v) for k, v in zip(PHASES, out[:7])}
    d["total"] = int(out[7])
    return d


def tobounds_checked() -> bool:
    return bool(lib().tobounds_checked())


def toget_bounds_report(problem, reset: bool = False) -> dict:
    """The problem's bounds-check report (checked build only; raises
    ToError TO_ERR_UNSUPPORTED in the release build)."""
    out = np.zeros(4, np.int64)
    _check(lib().toget_bounds_report(problem.handle, _ptr(out), int(reset)))
    return {"violations": int(out[0]), "site": int(out[1]), "index": int(out[2]), "limit": int(out[3])}


def tolast_launch_count(batch: Batch) -> int:
    return int(lib().tolast_launch_count(batch.handle))


class Solver:
    """One problem and a reusable batch: ``Solver(prob).solve(x0, T, ...)`` returns a result dict."""

    def __init__(self, prob, T_max=None, prec=TO_MIXED, B_max=None, knots_max=None, **opt_overrides):
        self.prob = prob
        self.T_max = int(T_max or 400)
        self.problem = tocreate_problem(prob.sys, prob.params, self.T_max, actor_w=prob.actor_w)
        self.opts = to_default_opts(prec=prec, **opt_overrides)
        self.batch = None
        self._cap = (0, 0, TO_MIXED)
        if B_max is not None:
            self._ensure(B_max, knots_max or B_max * (self.T_max + 1), prec)

    def _ensure(self, B, knots, prec):
        cB, cK, cP = self._cap
        if self.batch is None or B > cB or knots > cK or (prec == TO_FP64 and cP != TO_FP64):
            B, knots = max(B, cB), max(knots, cK)
            p = TO_FP64 if (prec == TO_FP64 or cP == TO_FP64) else TO_MIXED
            self.batch = None
            self.batch = tocreate_batch(self.problem, B, knots, to_default_opts(prec=p))
            self._cap = (B, knots, p)

    def solve(self, x0, T, U_init=None, forced_alpha=None, want=("X", "U"), history=True, **overrides):
        opts = to_default_opts(**{f: getattr(self.opts, f) for f, _ in to_solver_opts._fields_ if f != "forced_alpha"})
        for k, v in overrides.items():
            setattr(opts, k, v)
        Ts = np.broadcast_to(np.asarray(T), (np.atleast_2d(x0).shape[0],))
        self._ensure(len(Ts), int(np.sum(Ts + 1)), opts.prec)
        self.batch = tosolve_batch(self.problem, x0, T, U_init, opts, batch=self.batch, forced_alpha=forced_alpha)
        r = toget_trajectories(self.batch, X="X" in want, U="U" in want, Vx="Vx" in want, K="K" in want)
        if history:
            r["alpha_hist"], r["J_hist"] = toget_history(self.batch)
        return r
