"""ctypes binding of the plain FP64 CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package, and this package never imports the product library.

Every entry point follows the paper's statement of the method (Sec. II, Eq. 1
for the OCP; Sec. IV-A for the iteration budget; Sec. IV-B for eigenvalue
clipping); the C++ source cites each step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_CONVERGED, ST_MAX_ITER, ST_LS_FAIL, ST_NONFINITE, ST_FLAG_REG = 1, 2, 3, 4, 16


# plain g++, no arch flags; no FMA contraction, so every host (x86-64 or
# aarch64, where g++ contracts a*b+c by default) rounds each operation alike
_FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-pthread"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_lib/liboracle.so``."""
    os.makedirs(_LIBDIR, exist_ok=True)
    stamp = _SO + ".flags"
    old = open(stamp).read() if os.path.exists(stamp) else ""
    if (force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
            or old != " ".join(_FLAGS)):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["g++", *_FLAGS, _SRC, "-o", tmp], check=True)
        os.replace(tmp, _SO)
        with open(stamp, "w") as f:
            f.write(" ".join(_FLAGS))
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_SO)
    return _lib


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_F = C.POINTER(C.c_float)


def _d(a):
    return None if a is None else a.ctypes.data_as(_D)


def _i(a):
    return None if a is None else a.ctypes.data_as(_I)


def _f(a):
    return None if a is None else a.ctypes.data_as(_F)


def _arr(a, dt=np.float64):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


class Oracle:
    """Wraps one problem (system id + flat parameter vector + optional actor weights)."""

    def __init__(self, sys: int, params, actor_w=None):
        self.sys = int(sys)
        self.p = _arr(params)
        self.np = int(self.p.size)
        self.actor_w = _arr(actor_w, np.float32)
        n, m = C.c_int(), C.c_int()
        if lib().oracle_dims(self.sys, _d(self.p), self.np, C.byref(n), C.byref(m)) != 0:
            raise ValueError("oracle: malformed problem parameters")
        self.n, self.m = n.value, m.value

    @classmethod
    def from_problem(cls, prob):
        return cls(prob.sys, prob.params, prob.actor_w)

    def _call(self, name, *args):
        rc = getattr(lib(), name)(self.sys, _d(self.p), self.np, *args)
        if rc < 0:
            raise RuntimeError(f"oracle: {name} failed ({rc})")
        return rc

    # --- single evaluations -------------------------------------------------
    def step(self, x, u):
        x, u = _arr(x), _arr(u)
        xn = np.empty(self.n)
        self._call("oracle_step", _d(x), _d(u), _d(xn))
        return xn

    def linearize(self, x, u):
        x, u = _arr(x), _arr(u)
        A = np.empty((self.n, self.n))
        B = np.empty((self.n, self.m))
        self._call("oracle_linearize", _d(x), _d(u), _d(A), _d(B))
        return A, B

    def cost(self, x, u=None, terminal=False):
        """(l, gradient, Hessian) over z = [x; u] (terminal: z = x)."""
        x = _arr(x)
        u = _arr(np.zeros(self.m) if u is None else u)
        nz = self.n if terminal else self.n + self.m
        l = C.c_double()
        g = np.empty(nz)
        H = np.empty((nz, nz))
        self._call("oracle_cost", _d(x), _d(u), int(terminal), C.byref(l), _d(g), _d(H))
        return l.value, g, H

    def cost_value(self, x, u=None, terminal=False):
        x = _arr(x)
        u = _arr(np.zeros(self.m) if u is None else u)
        l = C.c_double()
        self._call("oracle_cost_value", _d(x), _d(u), int(terminal), C.byref(l))
        return l.value

    def rnea(self, q, qd, qdd, gravity=True, contact=False):
        q, qd, qdd = _arr(q), _arr(qd), _arr(qdd)
        tau = np.empty(q.size)
        self._call("oracle_rnea", _d(q), _d(qd), _d(qdd), int(gravity), int(contact), _d(tau))
        return tau

    def mass_matrix(self, q):
        q = _arr(q)
        M = np.empty((q.size, q.size))
        self._call("oracle_mass_matrix", _d(q), _d(M))
        return M

    def forward_dynamics(self, q, qd, tau):
        q, qd, tau = _arr(q), _arr(qd), _arr(tau)
        qdd = np.empty(q.size)
        self._call("oracle_forward_dynamics", _d(q), _d(qd), _d(tau), _d(qdd))
        return qdd

    def point_world(self, q, body, pt):
        q, pt = _arr(q), _arr(pt)
        out = np.empty(3)
        E0 = np.empty((3, 3))
        self._call("oracle_point_world", _d(q), int(body), _d(pt), _d(out), _d(E0))
        return out, E0

    def rollout(self, x0, U):
        x0, U = _arr(x0), _arr(U)
        T = U.shape[0]
        X = np.empty((T + 1, self.n))
        J = C.c_double()
        self._call("oracle_rollout", T, _d(x0), _d(U), _d(X), C.byref(J))
        return X, J.value

    def critic_targets(self, X, U, K):
        """Partial K-step cost-to-go at every knot of one trajectory (T+1 values)."""
        X, U = _arr(X), _arr(U)
        T = U.shape[0]
        Vbar = np.empty(T + 1)
        self._call("oracle_critic_targets", T, int(K), _d(X), _d(U), _d(Vbar))
        return Vbar

    def backward(self, X, U, eps=1e-8):
        X, U = _arr(X), _arr(U)
        T = U.shape[0]
        K = np.empty((T, self.m, self.n))
        k = np.empty((T, self.m))
        Vx = np.empty((T + 1, self.n))
        rc = self._call("oracle_backward", T, _d(X), _d(U), C.c_double(eps), _d(K), _d(k), _d(Vx))
        return K, k, Vx, rc

    def forward_pass(self, X, U, K, k, alpha):
        X, U, K, k = _arr(X), _arr(U), _arr(K), _arr(k)
        T = U.shape[0]
        Xn = np.empty_like(X)
        Un = np.empty_like(U)
        J = C.c_double()
        self._call("oracle_forward_pass", T, _d(X), _d(U), _d(K), _d(k), C.c_double(alpha), _d(Xn), _d(Un),
                   C.byref(J))
        return Xn, Un, J.value

    def actor(self, x):
        if self.actor_w is None:
            raise ValueError("problem has no actor weights")
        x = _arr(x)
        u = np.empty(self.m)
        lib().oracle_actor(_f(self.actor_w), self.n, 256, 256, self.m, _d(x), _d(u))
        return u

    # --- the full iLQR over a batch ----------------------------------------
    def solve(self, x0, T, U_init=None, max_iter=100, tol=1e-8, eps=1e-8, n_alpha=8, alpha_decay=0.5,
              forced=None, threads=0, want_vx=False, want_K=False, use_actor=True, reg="clip"):
        """iLQR as stated in the paper (reg="clip": eigenvalue clipping, Sec. IV-B),
        or the standard Levenberg-Marquardt variant it compares against (reg="lm")."""
        x0 = _arr(np.atleast_2d(x0))
        B = x0.shape[0]
        T = _arr(np.broadcast_to(np.asarray(T), (B,)), np.int32)
        T_max = int(T.max())
        if U_init is not None:
            U_init = _arr(U_init)
            assert U_init.shape == (B, T_max, self.m)
        if forced is not None:
            forced = _arr(forced, np.int32)
            assert forced.shape == (B, max_iter)
        X = np.empty((B, T_max + 1, self.n))
        U = np.empty((B, T_max, self.m))
        J = np.empty(B)
        iters = np.empty(B, np.int32)
        status = np.empty(B, np.int32)
        Vx = np.empty((B, T_max + 1, self.n)) if want_vx else None
        K = np.empty((B, T_max, self.m, self.n)) if want_K else None
        ah = np.full((B, max_iter), -1, np.int32)
        Jh = np.full((B, max_iter + 1), np.nan)
        aw = self.actor_w if use_actor else None
        rc = lib().oracle_solve_batch(self.sys, _d(self.p), self.np, _f(aw), B, T_max, _d(x0), _i(T), _d(U_init),
                                      int(max_iter), C.c_double(tol), C.c_double(eps), int(n_alpha),
                                      C.c_double(alpha_decay), _i(forced), int(threads), _d(X), _d(U), _d(J),
                                      _i(iters), _i(status), _d(Vx), _d(K), _i(ah), _d(Jh), int(reg == "lm"))
        if rc != 0:
            raise RuntimeError(f"oracle_solve_batch failed ({rc})")
        return dict(X=X, U=U, J=J, iters=iters, status=status, Vx=Vx, K=K, alpha_hist=ah, J_hist=Jh, T=T)


def std_critic(weights, X):
    """The std-critic MLP (n_in -> 256 tanh -> 256 tanh -> 1 softplus) in
    float64 on rows of X (Sec. III-C's V^std)."""
    X = np.asarray(X, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    n_in = X.shape[1]
    o = 0
    W1 = w[o:o + 256 * n_in].reshape(256, n_in); o += 256 * n_in
    b1 = w[o:o + 256]; o += 256
    W2 = w[o:o + 256 * 256].reshape(256, 256); o += 256 * 256
    b2 = w[o:o + 256]; o += 256
    W3 = w[o:o + 256].reshape(1, 256); o += 256
    b3 = w[o:o + 1]
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    z = (h2 @ W3.T + b3)[:, 0]
    return np.logaddexp(0.0, z)                  # softplus


def rank_candidates(weights, X, N):
    """Indices (ascending) of the N candidates with the largest std-critic
    score, ties broken by the lower index (Sec. III-D), and the scores."""
    s = std_critic(weights, X)
    order = np.lexsort((np.arange(s.size), -s))  # score descending, then index
    return np.sort(order[:N]), s


def eigclip(Q, eps):
    Q = _arr(Q)
    n = Q.shape[0]
    out = np.empty_like(Q)
    lib().oracle_eigclip(n, _d(Q), C.c_double(eps), _d(out))
    return out


def eig(Q):
    Q = _arr(Q)
    n = Q.shape[0]
    S = np.empty(n)
    W = np.empty((n, n))
    lib().oracle_eig(n, _d(Q), _d(S), _d(W))
    return S, W


def chol_solve(Quu, b):
    Quu, b = _arr(Quu), _arr(b)
    x = np.empty_like(b)
    rc = lib().oracle_chol_solve(Quu.shape[0], _d(Quu), _d(b), _d(x))
    return x, rc
