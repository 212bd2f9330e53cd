"""Seeded synthetic workloads for the batched trajectory-optimisation path.

This module only draws random inputs (problem parameters, initial states,
horizons, actor weights) and lays them out in the flat parameter format that
``include/to.h`` documents.  It holds no part of the solver's arithmetic: the
dynamics, costs and the iLQR iteration are implemented separately by the CUDA
library and by the CPU oracle, and both read what this module writes.

Every generator uses numpy's PCG64 seeded from ``(seed, stream)`` so that the
problem, the batch and the actor weights of one seed are independent streams.

The systems follow the paper's experimental section (point mass, planar
manipulator, quadruped) at the sizes of the synthetic workloads:

* ``POINTMASS`` (1): n=4 [px,py,vx,vy], m=2, explicit Euler dt=0.05, T=50,
  three Gaussian obstacle bumps, terminal 50|p|^2+|v|^2.
* ``PLANAR3`` (2): planar 3-link arm, n=6, m=3, semi-implicit Euler dt=0.01,
  T uniform in [100,400], two end-effector bumps, terminal reaching cost.
* ``ARM7`` (3): 7-DoF serial arm (axes z,y,z,y,z,y,z), n=14, m=7, T=200.
* ``QUAD`` (4): floating base (6 virtual joints) + 4 legs x 3 joints,
  n=36, m=12, penalty-spring ground contact, actor-MLP warm start, T=100.
* ``DUBINS`` (5): jerk-controlled Dubins car [px,py,theta,v,a], u=[omega,jerk],
  explicit Euler dt=0.05, T=100, three Gaussian obstacle bumps, terminal
  50|p|^2 + v^2 + a^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

POINTMASS, PLANAR3, ARM7, QUAD, DUBINS = 1, 2, 3, 4, 5
SYSTEM_NAMES = {POINTMASS: "pointmass2d", PLANAR3: "planar3", ARM7: "arm7", QUAD: "quad18", DUBINS: "dubins"}
NM = {POINTMASS: (4, 2), PLANAR3: (6, 3), ARM7: (14, 7), QUAD: (36, 12), DUBINS: (5, 2)}

# joint types of the rigid-body tree format
RX, RY, RZ, PX, PY, PZ = 0, 1, 2, 3, 4, 5
RIGID_HEADER = 8      # dt, gx, gy, gz, N, a0, n_sub, 0
BODY_STRIDE = 16      # parent, jtype, off[3], mass, com[3], I[3], 4 x reserved

ACTOR_SIZES = (36, 256, 256, 12)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


@dataclass
class Problem:
    sys: int
    n: int
    m: int
    dt: float
    params: np.ndarray                      # float64, layout of include/to.h
    actor_w: np.ndarray | None = None       # float32, W1 b1 W2 b2 W3 b3 (row-major)
    meta: dict = field(default_factory=dict)

    @property
    def name(self) -> str:
        return SYSTEM_NAMES[self.sys]


@dataclass
class Batch:
    x0: np.ndarray          # [B, n] float64
    T: np.ndarray           # [B] int32
    U_init: np.ndarray | None = None   # [B, T_max, m] float64 or None


def _body(parent, jtype, off, mass, com, inertia):
    row = np.zeros(BODY_STRIDE)
    row[0] = parent
    row[1] = jtype
    row[2:5] = off
    row[5] = mass
    row[6:9] = com
    row[9:12] = inertia
    return row


def _rigid(dt, gvec, bodies, a0, cost_block, n_sub=1):
    hdr = np.zeros(RIGID_HEADER)
    hdr[0] = dt
    hdr[1:4] = gvec
    hdr[4] = len(bodies)
    hdr[5] = a0
    hdr[6] = n_sub       # semi-implicit Euler substeps of dt / n_sub per knot
    return np.concatenate([hdr] + list(bodies) + [np.asarray(cost_block, dtype=np.float64)])


def rigid_cost_offset(n_bodies: int) -> int:
    return RIGID_HEADER + BODY_STRIDE * n_bodies


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------

def pointmass(seed: int = 0, n_bumps: int = 3, bump_amp: float = 5.0) -> Problem:
    """Point-mass double integrator with Gaussian obstacle bumps."""
    r = _rng(seed, 0)
    centres = r.uniform(-1.0, 1.0, size=(n_bumps, 2))
    p = np.zeros(5 + 2 * n_bumps + 2)
    p[0] = 0.05          # dt
    p[1] = 0.5e-2        # control weight
    p[2] = bump_amp      # bump amplitude
    p[3] = 0.1           # bump sigma
    p[4] = n_bumps
    p[5:5 + 2 * n_bumps] = centres.ravel()
    p[5 + 2 * n_bumps] = 50.0   # terminal position weight
    p[6 + 2 * n_bumps] = 1.0    # terminal velocity weight
    return Problem(POINTMASS, 4, 2, 0.05, p, meta={"centres": centres})


def dubins(seed: int = 0, n_bumps: int = 3, bump_amp: float = 5.0) -> Problem:
    """Jerk-controlled Dubins car with Gaussian obstacle bumps (the time state
    of the paper's version is dropped: every solve starts at t = 0)."""
    r = _rng(seed, 0)
    centres = r.uniform(-1.0, 1.0, size=(n_bumps, 2))
    p = np.zeros(5 + 2 * n_bumps + 3)
    p[0] = 0.05          # dt
    p[1] = 0.5e-2        # control weight
    p[2] = bump_amp      # bump amplitude
    p[3] = 0.1           # bump sigma
    p[4] = n_bumps
    p[5:5 + 2 * n_bumps] = centres.ravel()
    p[5 + 2 * n_bumps] = 50.0   # terminal position weight
    p[6 + 2 * n_bumps] = 1.0    # terminal speed weight
    p[7 + 2 * n_bumps] = 1.0    # terminal acceleration weight
    return Problem(DUBINS, 5, 2, 0.05, p, meta={"centres": centres})


def planar3(seed: int = 0, n_bumps: int = 2, bump_amp: float = 5.0) -> Problem:
    """Planar 3-link arm in a vertical plane, gravity along -y, joints about z."""
    r = _rng(seed, 0)
    L = r.uniform(0.5, 1.5, size=3)
    M = r.uniform(0.5, 1.5, size=3)
    reach = 0.8 * L.sum()

    def disk(k):
        rad = reach * np.sqrt(r.uniform(0.0, 1.0, size=k))
        ang = r.uniform(-math.pi, math.pi, size=k)
        return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)

    target = disk(1)[0]
    centres = disk(n_bumps)
    bodies = []
    for i in range(3):
        off = (0.0, 0.0, 0.0) if i == 0 else (L[i - 1], 0.0, 0.0)
        izz = M[i] * L[i] ** 2 / 12.0
        bodies.append(_body(i - 1, RZ, off, M[i], (L[i] / 2, 0.0, 0.0), (0.0, izz, izz)))
    cost = np.zeros(16)
    cost[0] = 1e-3            # torque weight
    cost[1] = bump_amp
    cost[2] = 0.1
    cost[3] = n_bumps
    cost[4:4 + 2 * n_bumps] = centres.ravel()
    cost[8:10] = target
    cost[10] = 100.0          # terminal end-effector weight
    cost[11] = 1.0            # terminal velocity weight
    cost[12] = 2              # end-effector body
    cost[13:16] = (L[2], 0.0, 0.0)
    p = _rigid(0.01, (0.0, -9.81, 0.0), bodies, 0, cost)
    return Problem(PLANAR3, 6, 3, 0.01, p, meta={"L": L, "M": M, "target": target, "centres": centres})


def arm7(seed: int = 0) -> Problem:
    """7-DoF serial arm, revolute axes z,y,z,y,z,y,z, links along the local -z
    (the chain hangs under gravity at q = 0)."""
    r = _rng(seed, 0)
    L = r.uniform(0.2, 0.6, size=7)
    M = r.uniform(0.5, 3.0, size=7)
    f = r.uniform(0.5, 1.5, size=(7, 3))
    reach = 0.8 * L.sum()
    d = r.normal(size=3)
    d /= np.linalg.norm(d)
    target = d * reach * r.uniform(0.0, 1.0) ** (1.0 / 3.0)
    axes = [RZ, RY, RZ, RY, RZ, RY, RZ]
    bodies = []
    for i in range(7):
        off = (0.0, 0.0, 0.0) if i == 0 else (0.0, 0.0, -L[i - 1])
        rod = M[i] * L[i] ** 2 / 12.0
        inertia = (f[i, 0] * rod, f[i, 1] * rod, f[i, 2] * rod)
        bodies.append(_body(i - 1, axes[i], off, M[i], (0.0, 0.0, -L[i] / 2), inertia))
    cost = np.zeros(11)
    cost[0] = 1e-4            # torque weight
    cost[1] = 1e-2            # running joint-velocity weight
    cost[2:5] = target
    cost[5] = 100.0           # terminal end-effector weight
    cost[6] = 1.0             # terminal velocity weight
    cost[7] = 6
    cost[8:11] = (0.0, 0.0, -L[6])
    p = _rigid(0.01, (0.0, 0.0, -9.81), bodies, 0, cost)
    return Problem(ARM7, 14, 7, 0.01, p, meta={"L": L, "M": M, "target": target})


QUAD_FEET = 4


def quad(seed: int = 0, with_actor: bool = True) -> Problem:
    """Floating base (Px,Py,Pz,Rz,Ry,Rx virtual joints) + 4 legs (hip x, thigh y, calf y)."""
    r = _rng(seed, 0)
    base_m = r.uniform(10.0, 12.0)
    bx, by, bz = 0.6, 0.3, 0.15
    base_I = (base_m * (by ** 2 + bz ** 2) / 12.0,
              base_m * (bx ** 2 + bz ** 2) / 12.0,
              base_m * (bx ** 2 + by ** 2) / 12.0)
    link_m = r.uniform(0.2, 2.0, size=(4, 3))
    link_l = r.uniform(0.2, 0.25, size=(4, 2))        # thigh, calf
    theta = r.uniform(0.5, 0.8)                       # nominal thigh angle; calf = -2 theta
    bodies = []
    for j, jt in enumerate([PX, PY, PZ, RZ, RY, RX]):
        if j < 5:
            bodies.append(_body(j - 1, jt, (0, 0, 0), 0.0, (0, 0, 0), (0, 0, 0)))
        else:
            bodies.append(_body(j - 1, jt, (0, 0, 0), base_m, (0, 0, 0), base_I))
    hips = [(+bx / 2, +by / 2), (+bx / 2, -by / 2), (-bx / 2, +by / 2), (-bx / 2, -by / 2)]
    feet = []
    for leg in range(4):
        hx, hy = hips[leg]
        mh, mt, mc = link_m[leg]
        lt, lc = link_l[leg]
        hip = len(bodies)
        # hip link: a short 5 cm block at the hip joint
        bodies.append(_body(5, RX, (hx, hy, 0.0), mh, (0.0, 0.0, 0.0),
                            (mh * 0.05 ** 2 / 6.0,) * 3))
        thigh = len(bodies)
        bodies.append(_body(hip, RY, (0.0, 0.0, 0.0), mt, (0.0, 0.0, -lt / 2),
                            (mt * lt ** 2 / 12.0, mt * lt ** 2 / 12.0, mt * 0.03 ** 2 / 2.0)))
        calf = len(bodies)
        bodies.append(_body(thigh, RY, (0.0, 0.0, -lt), mc, (0.0, 0.0, -lc / 2),
                            (mc * lc ** 2 / 12.0, mc * lc ** 2 / 12.0, mc * 0.02 ** 2 / 2.0)))
        feet.append((calf, (0.0, 0.0, -lc)))
    depth = float(np.mean((link_l[:, 0] + link_l[:, 1]) * math.cos(theta)))
    total_m = base_m + link_m.sum()
    z_nom = depth - (total_m * 9.81 / 4.0) / 1e4     # feet pressed in by the weight share
    cost = np.zeros(11 + 4 * QUAD_FEET)
    cost[0] = 1e-3            # torque weight
    cost[1] = z_nom
    cost[2] = 10.0            # base height weight
    cost[3] = 1.0             # base orientation weight
    cost[4] = 1.0             # forward velocity weight
    cost[5] = 0.5             # forward velocity target [m/s]
    cost[6] = 10.0            # terminal scale of the state terms
    cost[7] = 1e4             # contact stiffness
    cost[8] = 1e2             # contact damping
    cost[9] = 200.0           # softplus sharpness beta [1/m]
    cost[10] = QUAD_FEET
    for i, (b, pt) in enumerate(feet):
        cost[11 + 4 * i] = b
        cost[12 + 4 * i:15 + 4 * i] = pt
    # ten 1 ms substeps per 10 ms knot: the contact damper (1e2 N s/m) acting on
    # feet whose effective mass falls to ~0.05 kg needs dt_sub * d / m < 2
    p = _rigid(0.01, (0.0, 0.0, -9.81), bodies, 6, cost, n_sub=10)
    prob = Problem(QUAD, 36, 12, 0.01, p,
                   meta={"z_nom": z_nom, "theta": theta, "link_l": link_l, "link_m": link_m})
    if with_actor:
        prob.actor_w = actor_weights(seed)
    return prob


def actor_weights(seed: int, sizes=ACTOR_SIZES) -> np.ndarray:
    """PyTorch-style uniform(+-1/sqrt(fan_in)) init of W1,b1,W2,b2,W3,b3 (float32)."""
    r = _rng(seed, 7)
    parts = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        bound = 1.0 / math.sqrt(fi)
        parts.append(r.uniform(-bound, bound, size=(fo, fi)).ravel())
        parts.append(r.uniform(-bound, bound, size=fo))
    return np.concatenate(parts).astype(np.float32)


def std_critic_weights(n_in: int, seed: int = 0) -> np.ndarray:
    """Seeded std-critic MLP n_in -> 256 -> 256 -> 1 (same init as the actor;
    random weights: the ranking's cost, not its meaning)."""
    r = _rng(seed, 8)
    parts = []
    sizes = (n_in, 256, 256, 1)
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        bound = 1.0 / math.sqrt(fi)
        parts.append(r.uniform(-bound, bound, size=(fo, fi)).ravel())
        parts.append(r.uniform(-bound, bound, size=fo))
    return np.concatenate(parts).astype(np.float32)


def actor_param_count(sizes=ACTOR_SIZES) -> int:
    return sum(fo * fi + fo for fi, fo in zip(sizes[:-1], sizes[1:]))


def make_problem(sys: int, seed: int = 0, **kw) -> Problem:
    return {POINTMASS: pointmass, PLANAR3: planar3, ARM7: arm7, QUAD: quad, DUBINS: dubins}[sys](seed, **kw)


# --------------------------------------------------------------------------
# batches of initial states and horizons
# --------------------------------------------------------------------------

def make_batch(prob: Problem, B: int, seed: int = 0, T: int | tuple | None = None) -> Batch:
    """Initial states and horizons.  ``T`` may be an int, a (lo, hi) range or None (default)."""
    r = _rng(seed, 1)
    n = prob.n
    x0 = np.zeros((B, n))
    if prob.sys == POINTMASS:
        x0[:, 0:2] = r.uniform(-2.0, 2.0, size=(B, 2))
        Td = 50
    elif prob.sys == PLANAR3:
        x0[:, 0:3] = r.uniform(-math.pi, math.pi, size=(B, 3))
        Td = (100, 400)
    elif prob.sys == ARM7:
        x0[:, 0:7] = r.normal(0.0, 0.5, size=(B, 7))
        Td = 200
    elif prob.sys == QUAD:
        th = prob.meta["theta"]
        x0[:, 2] = prob.meta["z_nom"] + r.uniform(-0.05, 0.05, size=B)
        nominal = np.tile([0.0, th, -2.0 * th], 4)
        x0[:, 6:18] = nominal + r.uniform(-0.2, 0.2, size=(B, 12))
        Td = 100
    elif prob.sys == DUBINS:
        # position in the obstacle field's square, any heading, at rest
        x0[:, 0:2] = r.uniform(-2.0, 2.0, size=(B, 2))
        x0[:, 2] = r.uniform(-math.pi, math.pi, size=B)
        Td = 100
    else:
        raise ValueError(prob.sys)
    if T is None:
        T = Td
    if isinstance(T, tuple):
        Ts = r.integers(T[0], T[1] + 1, size=B).astype(np.int32)
    else:
        Ts = np.full(B, int(T), dtype=np.int32)
    return Batch(x0, Ts)


def serving_stream(rate: float, duration_s: float, seed: int = 0, systems=(POINTMASS, PLANAR3, ARM7),
                   T_range=(50, 400)):
    """Poisson arrivals: list of (t_arrival_s, sys, T, x0) with the system uniform over ``systems``."""
    r = _rng(seed, 3)
    t = 0.0
    out = []
    probs = {s: make_problem(s, seed) for s in systems}
    while True:
        t += r.exponential(1.0 / rate)
        if t >= duration_s:
            break
        s = systems[int(r.integers(0, len(systems)))]
        Tk = int(r.integers(T_range[0], T_range[1] + 1))
        b = make_batch(probs[s], 1, seed=int(r.integers(0, 2 ** 31)), T=Tk)
        out.append((t, s, Tk, b.x0[0]))
    return out
