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

Rigid-body trees (7-DoF arm, quadruped) are counted from their joint tree
(N bodies, parents first) with n_sub semi-implicit Euler substeps per knot;
per substep:

* Newton-Euler, per body, with single-axis joints: velocity 25, acceleration
  27, body force (two inertia products and three cross products) 96, force
  back to the parent 27, joint transform 2 -> 177; the quadruped adds the
  world pose of every body (60) and the four feet's contact forces (80 each);
* composite-rigid-body mass matrix: 70 per non-root body (rotate and shift
  the composite inertia), 10 per body (F = I_c S), 24 per (body, ancestor)
  pair (one force transform);
* dense Cholesky N^3 / 3, two triangular solves 2 N^2, integration 4 N;
* one tangent direction (a state coordinate or a control) carried through
  the substep: twice the Newton-Euler work (product rule) plus the solve and
  the integration.
"""
from __future__ import annotations

import numpy as np

from .workload import ARM7, DUBINS, PLANAR3, POINTMASS, QUAD


def riccati_flops(n: int, m: int, refine: bool) -> int:
    f = 2 * n ** 3 + 2 * n * n * m + n * n * (n + 1) + 2 * m * n * n + 2 * m * m * n + 2 * n * n + 2 * n * m
    f += m ** 3 // 3 + 2 * m * m * (n + 1) + 2 * m * n * (n + 1) + 2 * m * n
    if refine:
        f += 4 * m * m * (n + 1)
    return f


def cholesky_fp64_flops(m: int) -> int:
    """The float64 share of a mixed-precision backward knot: the Q_uu
    Cholesky (m^3/3), its pivot tests and reciprocal pivots (m^2 + 2m)."""
    return m ** 3 // 3 + m * m + 2 * m


def mixed_fp64_fraction(sys: int, n: int, m: int, total_per_knot_iter: float) -> float:
    """Fraction of a mixed solve's algorithmic FLOPs that run in float64."""
    return cholesky_fp64_flops(m) / max(total_per_knot_iter, 1.0)


def effective_peak(f32: float, f64: float, p32: float, p64: float) -> float:
    """Peak FLOP rate of a mix of float32 and float64 work: the binding time
    is f32 / p32 + f64 / p64 (the two pipes do not overlap in the bound)."""
    return (f32 + f64) / (f32 / p32 + f64 / p64)


# (primal dynamics, one directional derivative of inverse dynamics incl. the
#  M^{-1} solve, one column of M^{-1}, clipped running-cost derivatives,
#  running cost + step)
_SYSTEM = {
    POINTMASS: dict(primal=0, tangent=0, minv=0, costd=60, cost_step=40),
    PLANAR3: dict(primal=277, tangent=252, minv=24, costd=280, cost_step=314),
    # Dubins car: closed-form A, B (sincos + 6), bump terms and 2x2 clip as
    # the point mass, running cost + step with the heading's sincos
    DUBINS: dict(primal=0, tangent=0, minv=0, costd=70, cost_step=55),
}


ACTOR_FLOPS_PER_KNOT = 2 * (36 * 256 + 256 * 256 + 256 * 12) + 2 * 256   # 36-256-256-12 MLP, tanh


def rigid_counts(params) -> dict:
    """Per-knot FLOPs of a rigid-body tree from its parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    N, n_sub = int(p[4]), max(int(p[6]), 1)
    parent = [int(p[8 + 16 * i]) for i in range(N)]
    depth = []
    for i in range(N):
        depth.append(0 if parent[i] < 0 else depth[parent[i]] + 1)
    pairs = sum(depth)
    roots = sum(1 for x in parent if x < 0)
    quad = N == 18
    rnea = 177 * N + (60 * N + 80 * 4 if quad else 0)
    crba = 70 * (N - roots) + 10 * N + 24 * pairs
    solve = 2 * N * N
    primal_sub = rnea + crba + N ** 3 // 3 + solve + 4 * N
    tangent_sub = 2 * rnea + solve + 4 * N
    return dict(N=N, n_sub=n_sub, primal=n_sub * primal_sub, tangent=n_sub * tangent_sub, costd=8 * N,
                cost=6 * N, rnea_sub=rnea)


def derivative_flops_minimal(sys: int, n: int, m: int, params=None) -> int:
    """A count of the derivative step that does not grow with the number of
    tangent directions, for the rigid trees: per substep, the analytic
    derivatives of inverse dynamics d ID / d(q, v) (Carpentier and Mansard,
    RSS 2018: both N x N matrices in O(N d) spatial operations, taken here as
    four Newton-Euler passes), M^-1 applied to their 2N columns and to the m
    torque columns (2 N^2 each, the factor is the primal's), and the chain
    rule through the substeps (the semi-implicit Euler step's Jacobian times
    the accumulated n x (n + m) one: three N x N blocks times N x (n + m),
    from the second substep on).  Other systems: as derivative_flops."""
    if sys not in (ARM7, QUAD):
        return derivative_flops(sys, n, m, params)
    c = rigid_counts(params)
    N, n_sub = c["N"], c["n_sub"]
    rnea = c["rnea_sub"]
    per_sub = 4 * rnea + (2 * N + m) * 2 * N * N + 4 * N
    chain = 3 * 2 * N * N * (n + m)
    return n_sub * per_sub + (n_sub - 1) * chain + c["costd"] + c["primal"]


def derivative_flops(sys: int, n: int, m: int, params=None) -> int:
    if sys in (ARM7, QUAD):
        c = rigid_counts(params)
        return c["primal"] + (n + m) * c["tangent"] + c["costd"]
    c = _SYSTEM[sys]
    if sys == POINTMASS:
        return c["costd"]
    if sys == DUBINS:
        return 8 + c["costd"]
    return c["primal"] + n * c["tangent"] + m * c["minv"] + c["costd"]


def rollout_flops(sys: int, n: int, m: int, params=None) -> int:
    if sys in (ARM7, QUAD):
        c = rigid_counts(params)
        return 2 * m * n + 3 * m + n + c["primal"] + c["cost"]
    return 2 * m * n + 3 * m + n + _SYSTEM[sys]["cost_step"]


def solve_flops(sys: int, n: int, m: int, T: np.ndarray, iters: np.ndarray, status: np.ndarray,
                alpha_hist: np.ndarray, lanes_per_round: int, n_alpha: int, refine: bool, params=None,
                actor: bool = False, minimal_derivs: bool = False) -> float:
    """Algorithmic FLOPs of one batched solve from its per-instance history
    (minimal_derivs: the derivative step by derivative_flops_minimal)."""
    T = np.asarray(T, dtype=np.float64)
    iters = np.asarray(iters)
    dflops = derivative_flops_minimal(sys, n, m, params) if minimal_derivs else derivative_flops(sys, n, m, params)
    bwd = riccati_flops(n, m, refine) + dflops
    ro = rollout_flops(sys, n, m, params)
    total = float(np.sum(T) * (ro + (ACTOR_FLOPS_PER_KNOT if actor else 0)))   # warm-start rollout
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


def fp64_factor_in_mixed(group_lanes: int, lm: bool = False) -> bool:
    """Whether a mixed solve factors every Q_uu in float64.  Groups of 2 to 31
    lanes with clipped Hessians factor in float32 and fall back to the float64
    factor only for a Q_uu with a pivot below 2^-10 of its largest diagonal
    entry (7e-6 of the backward knots on the planar-arm bench workload; not
    counted here); single-lane groups, whole-warp groups and the
    Levenberg-Marquardt variant factor in float64."""
    return lm or not (2 <= group_lanes < 32)


def solve_flops_fp64(m: int, T: np.ndarray, iters: np.ndarray, status: np.ndarray, group_lanes: int = 1,
                     lm: bool = False) -> float:
    """The float64 FLOPs of a mixed solve (one Cholesky of Q_uu per backward
    knot where the factor runs in float64, see fp64_factor_in_mixed)."""
    if not fp64_factor_in_mixed(group_lanes, lm):
        return 0.0
    T = np.asarray(T, dtype=np.float64)
    failed = (np.asarray(status) & 15) == 3
    return float(np.sum(T * (np.asarray(iters) + failed)) * cholesky_fp64_flops(m))
