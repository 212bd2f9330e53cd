"""Algorithmic floating-point work of one iLQR solve, for the roofline.

Counts are FP adds, multiplies and FMAs (an FMA counts 2; sqrt, rsqrt, sin,
cos and exp count 1 each) of the minimal formulation of each step, per knot:

* backward Riccati step (Sec. II; Sec. IV-B's clip excluded):
    V A (2n^3) + V B (2n^2 m) + A^T (V A) upper triangle (n^2 (n+1))
    + B^T V A (2 m n^2) + B^T V B (2 m^2 n) + Q_x, Q_u (2n^2 + 2nm)
    + Cholesky (m^3/3) + gain solves (2 m^2 (n+1))
    + one refinement step in mixed mode (residual 2 m^2 (n+1), solves 2 m^2 (n+1))
    + V_xx update upper triangle (2 m n (n+1)) + V_x update (2 m n)
* derivatives: one primal dynamics evaluation, n directional derivatives of
  inverse dynamics (each 2x the primal Newton-Euler pass plus an M^{-1}
  solve), m columns of M^{-1}, and the clipped running-cost derivatives;
* line search: per candidate step size and knot, the policy
  u^ = u + alpha k + K dx (2mn + 3m + n) and one cost + dynamics evaluation.

The per-system constants below are hand counts of those formulations (the
planar arm: world-frame Newton-Euler 111, closed-form CRBA 106, 3x3 Cholesky
12, solve 18, kinematics 27).
"""
from __future__ import annotations

import numpy as np

from .workload import ARM7, PLANAR3, POINTMASS, QUAD


def riccati_flops(n: int, m: int, refine: bool) -> int:
    f = 2 * n ** 3 + 2 * n * n * m + n * n * (n + 1) + 2 * m * n * n + 2 * m * m * n + 2 * n * n + 2 * n * m
    f += m ** 3 // 3 + 2 * m * m * (n + 1) + 2 * m * n * (n + 1) + 2 * m * n
    if refine:
        f += 4 * m * m * (n + 1)
    return f


# (primal dynamics, one directional derivative of inverse dynamics incl. the
#  M^{-1} solve, one column of M^{-1}, clipped running-cost derivatives,
#  running cost + step)
_SYSTEM = {
    POINTMASS: dict(primal=0, tangent=0, minv=0, costd=60, cost_step=40),
    PLANAR3: dict(primal=277, tangent=252, minv=24, costd=280, cost_step=314),
}


def derivative_flops(sys: int, n: int, m: int) -> int:
    c = _SYSTEM[sys]
    if sys == POINTMASS:
        return c["costd"]
    return c["primal"] + n * c["tangent"] + m * c["minv"] + c["costd"]


def rollout_flops(sys: int, n: int, m: int) -> int:
    return 2 * m * n + 3 * m + n + _SYSTEM[sys]["cost_step"]


def solve_flops(sys: int, n: int, m: int, T: np.ndarray, iters: np.ndarray, status: np.ndarray,
                alpha_hist: np.ndarray, lanes_per_round: int, n_alpha: int, refine: bool) -> float:
    """Algorithmic FLOPs of one batched solve from its per-instance history."""
    T = np.asarray(T, dtype=np.float64)
    iters = np.asarray(iters)
    bwd = riccati_flops(n, m, refine) + derivative_flops(sys, n, m)
    ro = rollout_flops(sys, n, m)
    total = float(np.sum(T) * ro)                       # warm-start rollout
    total += float(np.sum(T * iters) * bwd)             # one backward pass per iteration
    # candidates evaluated: lanes_per_round per round; an accepted index j
    # needs j // lanes_per_round + 1 rounds; a failed search runs every round
    rounds_all = -(-n_alpha // lanes_per_round)
    cand = np.zeros(len(T))
    for i in range(len(T)):
        a = alpha_hist[i, :iters[i]]
        cand[i] = np.sum(np.minimum(n_alpha, (a // lanes_per_round + 1) * lanes_per_round))
    # a run that ended in a failed line search did one more backward pass and
    # searched every round
    failed = (np.asarray(status) & 15) == 3
    cand = cand + failed * min(n_alpha, rounds_all * lanes_per_round)
    total += float(np.sum(T * failed) * bwd)
    total += float(np.sum(T * cand) * ro)
    return total
