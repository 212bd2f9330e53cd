"""Pins of the oracle's rigid-body dynamics against closed forms and mechanics.

None of these re-types the oracle's recursion: they compare it with textbook
closed forms (pendulum, two-link planar arm), with Lagrangian identities
evaluated by finite differences of the kinematics (kinetic energy, Christoffel
symbols, potential energy), with free fall and with momentum conservation.
"""
import math

import numpy as np
import pytest

from paper_2602_19699_gb300 import workload as W


def _rigid_planar(lengths, masses, g=9.81):
    bodies = []
    for i, (l, m) in enumerate(zip(lengths, masses)):
        off = (0.0, 0.0, 0.0) if i == 0 else (lengths[i - 1], 0.0, 0.0)
        izz = m * l * l / 12.0
        bodies.append(W._body(i - 1, W.RZ, off, m, (l / 2, 0, 0), (0.0, izz, izz)))
    N = len(lengths)
    cost = np.zeros(16)
    cost[12] = N - 1
    cost[13] = lengths[-1]
    return W._rigid(0.01, (0.0, -g, 0.0), bodies, 0, cost)


def _oracle(oracle_mod, sys, params):
    return oracle_mod.Oracle(sys, params)


def test_pendulum_closed_form(oracle_mod):
    l, m, g = 0.8, 1.3, 9.81
    o = _oracle(oracle_mod, W.PLANAR3, _rigid_planar([l], [m], g))
    for q, qd, tau in [(0.3, 0.0, 0.0), (-1.2, 2.0, 0.7), (2.5, -1.0, -3.0)]:
        qdd = o.forward_dynamics([q], [qd], [tau])[0]
        # joint angle from the +x axis, gravity along -y: I_O qdd = tau - m g (l/2) cos q
        expect = (tau - m * g * (l / 2) * math.cos(q)) / (m * l * l / 3.0)
        assert abs(qdd - expect) < 1e-12 * max(1.0, abs(expect))


def test_two_link_mass_matrix_closed_form(oracle_mod):
    l1, l2, m1, m2 = 0.9, 0.7, 1.1, 0.6
    o = _oracle(oracle_mod, W.PLANAR3, _rigid_planar([l1, l2], [m1, m2]))
    lc1, lc2 = l1 / 2, l2 / 2
    I1, I2 = m1 * l1 ** 2 / 12, m2 * l2 ** 2 / 12
    rng = np.random.default_rng(0)
    for _ in range(5):
        q = rng.uniform(-3, 3, 2)
        c2 = math.cos(q[1])
        # Spong, Hutchinson & Vidyasagar, Robot Modeling and Control, sec. 7.4
        m11 = m1 * lc1 ** 2 + m2 * (l1 ** 2 + lc2 ** 2 + 2 * l1 * lc2 * c2) + I1 + I2
        m12 = m2 * (lc2 ** 2 + l1 * lc2 * c2) + I2
        m22 = m2 * lc2 ** 2 + I2
        M = o.mass_matrix(q)
        np.testing.assert_allclose(M, [[m11, m12], [m12, m22]], rtol=1e-13, atol=1e-13)


def _rot_axis(ax, q):
    c, s = math.cos(q), math.sin(q)
    R = np.eye(3)
    i, j = (ax + 1) % 3, (ax + 2) % 3
    R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
    return R


def _fk_homogeneous(params, q):
    """World rotation (body->world) and origin of every body, composed as
    active rotations R = R_parent Rot(axis, q) (an independent formulation)."""
    N = int(params[4])
    Rs, ps = [], []
    for i in range(N):
        row = params[8 + 16 * i: 8 + 16 * (i + 1)]
        parent, jt = int(row[0]), int(row[1])
        off = row[2:5].copy()
        Rp = np.eye(3) if parent < 0 else Rs[parent]
        pp = np.zeros(3) if parent < 0 else ps[parent]
        if jt <= W.RZ:
            Rj, dj = _rot_axis(jt, q[i]), np.zeros(3)
        else:
            Rj, dj = np.eye(3), np.eye(3)[jt - W.PX] * q[i]
        ps.append(pp + Rp @ (off + dj))
        Rs.append(Rp @ Rj)
    return Rs, ps


@pytest.mark.parametrize("sysid", [W.PLANAR3, W.ARM7, W.QUAD])
def test_forward_kinematics_matches_homogeneous_chain(oracle_mod, sysid):
    prob = W.make_problem(sysid, seed=3)
    o = oracle_mod.Oracle(prob.sys, prob.params)
    N = o.n // 2
    rng = np.random.default_rng(1)
    q = rng.uniform(-1, 1, N)
    Rs, ps = _fk_homogeneous(prob.params, q)
    for b in range(N):
        pt = rng.uniform(-0.3, 0.3, 3)
        pw, E0 = o.point_world(q, b, pt)
        np.testing.assert_allclose(pw, ps[b] + Rs[b] @ pt, atol=1e-13)
        np.testing.assert_allclose(E0.T, Rs[b], atol=1e-13)


def _bodies(params):
    N = int(params[4])
    return [params[8 + 16 * i: 8 + 16 * (i + 1)] for i in range(N)]


def _kinetic_energy_fd(params, q, qd, h=1e-6):
    """sum 1/2 m |v_c|^2 + 1/2 w_b^T I w_b with v_c and w from central differences of the kinematics."""
    Rp, pp = _fk_homogeneous(params, q + h * qd)
    Rm, pm = _fk_homogeneous(params, q - h * qd)
    R0, _ = _fk_homogeneous(params, q)
    T = 0.0
    for i, row in enumerate(_bodies(params)):
        m, com, I = row[5], row[6:9], row[9:12]
        vc = ((pp[i] + Rp[i] @ com) - (pm[i] + Rm[i] @ com)) / (2 * h)
        Rdot = (Rp[i] - Rm[i]) / (2 * h)
        Wb = R0[i].T @ Rdot          # skew matrix of the body-frame angular velocity
        w = np.array([Wb[2, 1], Wb[0, 2], Wb[1, 0]])
        T += 0.5 * m * vc @ vc + 0.5 * w @ (I * w)
    return T


def _potential(params, q):
    g = params[1:4]
    Rs, ps = _fk_homogeneous(params, q)
    return -sum(row[5] * g @ (ps[i] + Rs[i] @ row[6:9]) for i, row in enumerate(_bodies(params)))


def _no_contact(params):
    p = params.copy()
    off = W.rigid_cost_offset(int(p[4]))
    p[off + 7] = 0.0    # stiffness
    p[off + 8] = 0.0    # damping
    return p


@pytest.mark.parametrize("sysid", [W.PLANAR3, W.ARM7, W.QUAD])
def test_mass_matrix_is_kinetic_energy_hessian(oracle_mod, sysid):
    prob = W.make_problem(sysid, seed=5)
    o = oracle_mod.Oracle(prob.sys, prob.params)
    N = o.n // 2
    rng = np.random.default_rng(2)
    q = rng.uniform(-1, 1, N)
    M = o.mass_matrix(q)
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > 0
    for _ in range(3):
        qd = rng.normal(size=N)
        T_fd = _kinetic_energy_fd(prob.params, q, qd)
        assert abs(0.5 * qd @ M @ qd - T_fd) < 1e-8 * max(1.0, T_fd)


@pytest.mark.parametrize("sysid", [W.PLANAR3, W.ARM7, W.QUAD])
def test_rnea_matches_lagrangian(oracle_mod, sysid):
    """h(q, qd) = C(q, qd) qd + dV/dq with Christoffel symbols of FD dM/dq."""
    prob = W.make_problem(sysid, seed=7)
    params = _no_contact(prob.params) if sysid == W.QUAD else prob.params
    o = oracle_mod.Oracle(prob.sys, params)
    N = o.n // 2
    rng = np.random.default_rng(3)
    q = rng.uniform(-1, 1, N)
    qd = rng.normal(size=N)
    h = 1e-5
    dM = np.zeros((N, N, N))           # dM[:, :, k] = dM/dq_k
    for k in range(N):
        e = np.zeros(N); e[k] = h
        dM[:, :, k] = (o.mass_matrix(q + e) - o.mass_matrix(q - e)) / (2 * h)
    # c_i = sum_jk Gamma_ijk qd_j qd_k, Gamma_ijk = 1/2 (dM_ij/dq_k + dM_ik/dq_j - dM_jk/dq_i)
    c = np.einsum("ijk,j,k->i", dM, qd, qd) - 0.5 * np.einsum("jki,j,k->i", dM, qd, qd)
    gq = np.array([(_potential(params, q + np.eye(N)[i] * h) - _potential(params, q - np.eye(N)[i] * h)) / (2 * h)
                   for i in range(N)])
    tau = o.rnea(q, qd, np.zeros(N), gravity=True, contact=False)
    scale = max(1.0, np.abs(tau).max())
    np.testing.assert_allclose(tau, c + gq, atol=1e-6 * scale)
    # gravity-free, velocity-free inverse dynamics is linear in the acceleration
    a = rng.normal(size=N)
    np.testing.assert_allclose(o.rnea(q, np.zeros(N), a, gravity=False), o.mass_matrix(q) @ a, atol=1e-11)


@pytest.mark.parametrize("sysid", [W.PLANAR3, W.ARM7, W.QUAD])
def test_forward_inverse_roundtrip(oracle_mod, sysid):
    prob = W.make_problem(sysid, seed=1)
    o = oracle_mod.Oracle(prob.sys, prob.params)
    N = o.n // 2
    rng = np.random.default_rng(4)
    q, qd, tau = rng.uniform(-1, 1, N), rng.normal(size=N), rng.normal(size=N)
    qdd = o.forward_dynamics(q, qd, tau)
    back = o.rnea(q, qd, qdd, gravity=True, contact=(sysid == W.QUAD))
    np.testing.assert_allclose(back, tau, atol=1e-9 * max(1, np.abs(tau).max()))


def test_quadruped_free_fall(oracle_mod):
    prob = W.quad(seed=2, with_actor=False)
    params = _no_contact(prob.params)
    o = oracle_mod.Oracle(W.QUAD, params)
    q = np.zeros(18)
    q[2] = 1.0
    q[6:] = np.random.default_rng(5).uniform(-0.5, 0.5, 12)
    qdd = o.forward_dynamics(q, np.zeros(18), np.zeros(18))
    expect = np.zeros(18)
    expect[2] = -9.81
    np.testing.assert_allclose(qdd, expect, atol=1e-10)


def test_quadruped_momentum_conserved_without_gravity_and_contact(oracle_mod):
    prob = W.quad(seed=4, with_actor=False)
    params = _no_contact(prob.params)
    params[1:4] = 0.0
    o = oracle_mod.Oracle(W.QUAD, params)
    rng = np.random.default_rng(6)
    q = rng.uniform(-0.5, 0.5, 18)
    qd = rng.normal(size=18)
    tau = np.concatenate([np.zeros(6), rng.normal(size=12)])   # base unactuated
    qdd = o.forward_dynamics(q, qd, tau)
    h = 1e-4
    qp = q + h * qd + 0.5 * h * h * qdd
    qm = q - h * qd + 0.5 * h * h * qdd
    Rp, pp = _fk_homogeneous(params, qp)
    Rm, pm = _fk_homogeneous(params, qm)
    R0, p0 = _fk_homogeneous(params, q)
    ftot = np.zeros(3)
    scale = 0.0
    for i, row in enumerate(_bodies(params)):
        m, com = row[5], row[6:9]
        ac = ((pp[i] + Rp[i] @ com) - 2 * (p0[i] + R0[i] @ com) + (pm[i] + Rm[i] @ com)) / (h * h)
        ftot += m * ac
        scale += m * np.abs(ac).sum()
    assert np.abs(ftot).max() < 1e-5 * max(scale, 1.0)


def test_quadruped_contact_force_direction(oracle_mod):
    """A foot pressed into the ground receives an upward force: the support
    torques on the base's vertical joint equal the summed normal forces."""
    prob = W.quad(seed=0, with_actor=False)
    o = oracle_mod.Oracle(W.QUAD, prob.params)
    th = prob.meta["theta"]
    q = np.zeros(18)
    q[6:] = np.tile([0.0, th, -2 * th], 4)
    q[2] = prob.meta["z_nom"] - 0.01
    with_c = o.rnea(q, np.zeros(18), np.zeros(18), gravity=False, contact=True)
    # RNEA returns M qdd + h - J^T F: the Pz row is minus the total vertical force
    off = W.rigid_cost_offset(18)
    k, beta = prob.params[off + 7], prob.params[off + 9]
    fz = 0.0
    for f in range(4):
        b = int(prob.params[off + 11 + 4 * f])
        pt = prob.params[off + 12 + 4 * f: off + 15 + 4 * f]
        z = o.point_world(q, b, pt)[0][2]
        fz += k * math.log1p(math.exp(-beta * z)) / beta
    assert fz > 0
    assert abs(-with_c[2] - fz) < 1e-9 * fz


def test_dubins_closed_forms(oracle_mod):
    """Explicit-Euler Dubins car: a constant turn rate at constant speed sums
    a geometric series of headings (Sum_k cos(a + k d) = sin(K d / 2) /
    sin(d / 2) cos(a + (K - 1) d / 2)); a constant jerk integrates twice to
    v_K = v_0 + K dt a_0 + dt^2 j K (K - 1) / 2."""
    prob = W.dubins(seed=1)
    o = oracle_mod.Oracle.from_problem(prob)
    dt = prob.params[0]
    th0, v, om, K = 0.3, 1.7, 0.9, 40
    x = np.array([0.2, -0.4, th0, v, 0.0])
    for _ in range(K):
        x = o.step(x, np.array([om, 0.0]))
    d = dt * om
    g = np.sin(K * d / 2) / np.sin(d / 2)
    px = 0.2 + dt * v * g * np.cos(th0 + (K - 1) * d / 2)
    py = -0.4 + dt * v * g * np.sin(th0 + (K - 1) * d / 2)
    np.testing.assert_allclose(x[:3], [px, py, th0 + K * d], rtol=1e-12, atol=1e-12)
    assert x[3] == pytest.approx(v, rel=1e-15)
    a0, j = 0.3, -0.8
    x = np.array([0.0, 0.0, 0.0, 0.5, a0])
    for _ in range(K):
        x = o.step(x, np.array([0.0, j]))
    assert x[3] == pytest.approx(0.5 + K * dt * a0 + dt * dt * j * K * (K - 1) / 2, rel=1e-12)
    assert x[4] == pytest.approx(a0 + K * dt * j, rel=1e-12)
