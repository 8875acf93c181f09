"""Pins of the FP64 oracle against closed forms, invariants and special cases.

None of these tests re-types an oracle formula: each checks a consequence the paper's
equations fix (a free-fall trajectory, an exact conservation identity, a symmetric
special case, a textbook solution, brute force on a tiny input), chosen so that a
dropped term, a wrong sign, a transposed rotation or a swapped index fails one.
CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)
MAXRPM = oracle.max_rpm(P)
DT = P.dt_sim


# ---- small, independent quaternion helpers written for the tests ----
def qmul(a, b):
    """Hamilton product via the 4x4 left-multiplication matrix (a different route from the oracle)."""
    w, x, y, z = a
    L = np.array([[w, -x, -y, -z], [x, w, -z, y], [y, z, w, -x], [z, -y, x, w]], dtype=float)
    return L @ np.asarray(b, dtype=float)


def qconj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])


def axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=float)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])


def state(p=(0, 0, 1), q=(1, 0, 0, 0), v=(0, 0, 0), w=(0, 0, 0)):
    return np.concatenate([p, q, v, w]).astype(float)


def run_substeps(params, x, rpm, flags, k, dt=None):
    x = np.atleast_2d(np.asarray(x, dtype=float))
    rpm = np.atleast_2d(np.asarray(rpm, dtype=float))
    for _ in range(k):
        x = oracle.substep(params, x, rpm, flags, dt)
    return x


# ---------------------------------------------------------------- constants
def test_constants_match_paper_tables(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "cf2x_paper_constants.json")))
    d = P.to_dict()
    for k, v in g.items():
        if k.startswith("_"):
            continue
        np.testing.assert_allclose(d[k], v["value"], rtol=1e-15, err_msg=k)


def test_max_rpm_is_thrust_to_weight_times_weight():
    # Four rotors at MAX_RPM lift thrust2weight times the weight.
    T, _ = oracle.motor(P, [MAXRPM] * 4)
    assert T == pytest.approx(P.thrust2weight * P.mass * P.g, rel=1e-14)
    assert MAXRPM / HOVER == pytest.approx(math.sqrt(P.thrust2weight), rel=1e-14)


# ---------------------------------------------------------------- motor / hover
def test_hover_rpm_holds_altitude():
    x = run_substeps(P, state(p=(0.3, -0.2, 1.0)), [HOVER] * 4, 0, 1000)[0]
    assert abs(x[2] - 1.0) < 1e-9
    assert np.all(np.abs(x[7:10]) < 1e-9)
    np.testing.assert_allclose(x[3:7], [1, 0, 0, 0], atol=1e-15)


def test_motor_mixing_special_cases():
    n = 15000.0
    T, tau = oracle.motor(P, [n, n, n, n])
    assert np.all(np.abs(tau) < 1e-22)
    # one rotor at a time: the X-configuration signs of Eq. motor
    l = P.arm / math.sqrt(2)
    signs = {0: (1, -1, -1), 1: (1, 1, 1), 2: (-1, 1, -1), 3: (-1, -1, 1)}
    for i, (sx, sy, sz) in signs.items():
        r = [0.0] * 4
        r[i] = n
        T, tau = oracle.motor(P, r)
        F = P.kf * n * n
        assert T == pytest.approx(F, rel=1e-15)
        assert tau[0] == pytest.approx(sx * l * F, rel=1e-14)
        assert tau[1] == pytest.approx(sy * l * F, rel=1e-14)
        assert tau[2] == pytest.approx(sz * P.km * n * n, rel=1e-14)


def test_allocation_matrix_inverts_the_motor_model():
    # M applied to k_f n^2 reproduces [T, tau] of Eq. motor for arbitrary RPMs.
    rng = np.random.default_rng(0)
    M = oracle.allocation_matrix(P)
    for _ in range(20):
        r = rng.uniform(0, MAXRPM, 4)
        T, tau = oracle.motor(P, r)
        np.testing.assert_allclose(M @ (P.kf * r * r), np.concatenate([[T], tau]), rtol=1e-12, atol=1e-20)


# ---------------------------------------------------------------- translation
def test_free_fall_is_exact_forward_euler():
    # n = 0: v_k = -g dt k and z_k = z0 - g dt^2 k(k-1)/2 (forward Euler: p uses the old v).
    z0, K = 2.0, 240
    x = np.atleast_2d(state(p=(0, 0, z0)))
    for k in range(1, K + 1):
        x = oracle.substep(P, x, np.zeros((1, 4)), 0)
        assert x[0, 9] == pytest.approx(-P.g * DT * k, rel=1e-13)
        assert x[0, 2] == pytest.approx(z0 - P.g * DT * DT * k * (k - 1) / 2, rel=1e-13, abs=1e-13)
    # against the continuous solution the error is +g t dt / 2
    t = K * DT
    assert x[0, 2] - (z0 - 0.5 * P.g * t * t) == pytest.approx(P.g * t * DT / 2, rel=1e-9)


@pytest.mark.parametrize("axis,ang", [((1, 0, 0), 0.3), ((0, 1, 0), -0.4), ((1, 1, 0), 0.2)])
def test_thrust_points_along_body_z_in_world(axis, ang):
    # Hover RPM on a tilted drone: one substep from rest gives v = dt (g R e_z - g e_z),
    # with R e_z computed by the quaternion sandwich q (0, e_z) q*.
    q = axis_angle(axis, ang)
    bz = qmul(qmul(q, [0, 0, 0, 1]), qconj(q))[1:]
    x = run_substeps(P, state(q=q), [HOVER] * 4, 0, 1)[0]
    np.testing.assert_allclose(x[7:10], DT * P.g * (bz - np.array([0, 0, 1])), rtol=1e-12, atol=1e-15)


def test_rotation_matrix_matches_quaternion_sandwich():
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        R = oracle.rotation(q)
        for e in np.eye(3):
            np.testing.assert_allclose(R @ e, qmul(qmul(q, np.concatenate([[0], e])), qconj(q))[1:], atol=1e-14)


def test_quat_mul_basis_table():
    one, i, j, k = np.eye(4)
    np.testing.assert_allclose(oracle.quat_mul(i, j), k)
    np.testing.assert_allclose(oracle.quat_mul(j, k), i)
    np.testing.assert_allclose(oracle.quat_mul(k, i), j)
    np.testing.assert_allclose(oracle.quat_mul(i, i), -one)
    np.testing.assert_allclose(oracle.quat_mul(j, i), -k)


def test_rpy_inverts_zyx_composition():
    rng = np.random.default_rng(2)
    for _ in range(50):
        r, p, y = rng.uniform(-3.0, 3.0), rng.uniform(-1.5, 1.5), rng.uniform(-3.0, 3.0)
        q = qmul(qmul(axis_angle((0, 0, 1), y), axis_angle((0, 1, 0), p)), axis_angle((1, 0, 0), r))
        np.testing.assert_allclose(oracle.rpy(q), [r, p, y], atol=1e-12)


# ---------------------------------------------------------------- rotation dynamics
def test_principal_axis_spin_is_exact():
    w = 7.0
    x = np.atleast_2d(state(w=(0, 0, w)))
    for k in range(1, 101):
        x = oracle.substep(P, x, np.full((1, 4), HOVER), 0)
        np.testing.assert_array_equal(x[0, 10:13], [0, 0, w])
        ang = w * k * DT
        np.testing.assert_allclose(x[0, 3:7], [math.cos(ang / 2), 0, 0, math.sin(ang / 2)], atol=1e-13)
    assert oracle.rpy(x[0, 3:7])[2] == pytest.approx(w * 100 * DT, abs=1e-12)


def test_exp_map_is_exact_for_constant_body_rate():
    # Spherical inertia: omega stays constant under zero torque, so q_k = q0 (x) exp(k dt omega / 2).
    Ps = oracle.cf2x()
    Ps.Jxx = Ps.Jyy = Ps.Jzz = 2e-5
    rng = np.random.default_rng(3)
    q0 = rng.normal(size=4)
    q0 /= np.linalg.norm(q0)
    w = np.array([3.0, -5.0, 2.0])
    x = run_substeps(Ps, state(q=q0, w=w), [HOVER] * 4, 0, 50)[0]
    nw = np.linalg.norm(w)
    expect = qmul(q0, axis_angle(w, nw * 50 * DT))
    np.testing.assert_allclose(x[3:7], expect, atol=1e-12)
    np.testing.assert_allclose(x[10:13], w, rtol=1e-15)
    assert np.linalg.norm(x[3:7]) == pytest.approx(1.0, abs=1e-15)


def test_forward_euler_angular_momentum_identity():
    # Zero torque, L = J omega in the body frame: forward Euler gives exactly
    # |L_{k+1}|^2 = |L_k|^2 + dt^2 |omega_k x L_k|^2.
    J = np.array([P.Jxx, P.Jyy, P.Jzz])
    x = np.atleast_2d(state(w=(4.0, -3.0, 9.0)))
    for _ in range(20):
        w = x[0, 10:13]
        L = J * w
        x = oracle.substep(P, x, np.full((1, 4), HOVER), 0)
        L1 = J * x[0, 10:13]
        lhs = L1 @ L1
        rhs = L @ L + DT * DT * np.cross(w, L) @ np.cross(w, L)
        assert lhs == pytest.approx(rhs, rel=1e-13)


def test_symmetric_top_matches_textbook_solution():
    # Jxx = Jyy: body rates precess at lambda = (Jzz - Jxx)/Jxx * w_z
    # (w_x + i w_y)(t) = (w_x0 + i w_y0) exp(i lambda t). Forward Euler converges at O(dt).
    Ps = oracle.cf2x()
    Ps.dt_sim = 1e-5
    wx0, wy0, wz = 1.5, -0.5, 10.0
    K = 50000
    env_off = np.array([0, 1], dtype=np.int32)
    x, _, _ = oracle.control_steps(Ps, env_off, [0], [oracle.ACT_RPM], state(w=(wx0, wy0, wz))[None],
                                   np.zeros((1, 6)), np.zeros((1, 4)), np.full((1, 1, 4), HOVER), K)
    t = K * Ps.dt_sim
    lam = (Ps.Jzz - Ps.Jxx) / Ps.Jxx * wz
    c = (wx0 + 1j * wy0) * np.exp(1j * lam * t)
    np.testing.assert_allclose(x[0, 10:12], [c.real, c.imag], rtol=1e-3, atol=1e-4)
    assert x[0, 12] == pytest.approx(wz, rel=1e-14)


# ---------------------------------------------------------------- ground effect
def _extra_fz(params, x, rpm, flag):
    F1, _ = oracle.env_forces(params, np.atleast_2d(x), np.atleast_2d(rpm), flag)
    F0, _ = oracle.env_forces(params, np.atleast_2d(x), np.atleast_2d(rpm), 0)
    return F1[0] - F0[0]


def test_ground_effect_scaling_laws():
    r = [HOVER] * 4
    T, _ = oracle.motor(P, r)
    # inverse-square law in h above the clip height, ratio to thrust independent of RPM
    d1 = _extra_fz(P, state(p=(0, 0, 0.05)), r, oracle.GND)
    d2 = _extra_fz(P, state(p=(0, 0, 0.10)), r, oracle.GND)
    assert d1[2] / d2[2] == pytest.approx(4.0, rel=1e-13)
    assert d1[0] == 0 and d1[1] == 0
    r2 = [1.3 * HOVER] * 4
    T2, _ = oracle.motor(P, r2)
    e1 = _extra_fz(P, state(p=(0, 0, 0.05)), r2, oracle.GND)
    assert e1[2] / T2 == pytest.approx(d1[2] / T, rel=1e-13)
    # constant below the clip height (also for negative z)
    lo = [_extra_fz(P, state(p=(0, 0, h)), r, oracle.GND)[2] for h in (P.h_clip, 0.5 * P.h_clip, 0.0, -1.0)]
    assert np.ptp(lo) == 0.0 and lo[0] > 0


def test_ground_effect_doubles_thrust_at_special_height():
    # At h* = (r_p/4) sqrt(C_gnd) the increment equals the thrust itself, so a level drone
    # at hover RPM accelerates upward at exactly g.
    h = 0.25 * P.prop_radius * math.sqrt(P.c_gnd)
    assert h > P.h_clip
    F, _ = oracle.env_forces(P, state(p=(0, 0, h))[None], np.full((1, 4), HOVER), oracle.GND)
    assert F[0, 2] / P.mass == pytest.approx(P.g, rel=1e-12)


@pytest.mark.parametrize("roll,on", [(0.0, True), (1.5, True), (-1.5, True), (1.65, False), (3.0, False)])
def test_ground_effect_gate_on_roll(roll, on):
    d = _extra_fz(P, state(p=(0, 0, 0.05), q=axis_angle((1, 0, 0), roll)), [HOVER] * 4, oracle.GND)
    assert (d[2] > 0) == on


def test_ground_effect_gate_on_pitch():
    assert _extra_fz(P, state(p=(0, 0, 0.05), q=axis_angle((0, 1, 0), 1.5)), [HOVER] * 4, oracle.GND)[2] > 0
    # pitch beyond pi/2 is represented by roll = yaw = pi, pitch < pi/2 in ZYX: the body is inverted
    assert _extra_fz(P, state(p=(0, 0, 0.05), q=axis_angle((0, 1, 0), 1.7)), [HOVER] * 4, oracle.GND)[2] == 0


# ---------------------------------------------------------------- drag
def test_drag_level_special_case_and_axes():
    r = np.array([HOVER, 1.1 * HOVER, 0.9 * HOVER, HOVER])
    k = 2 * math.pi / 60 * r.sum()
    d = _extra_fz(P, state(v=(2.0, 0, 0)), r, oracle.DRAG)
    np.testing.assert_allclose(d, [-P.c_xy * k * 2.0, 0, 0], rtol=1e-13, atol=1e-20)
    d = _extra_fz(P, state(v=(0, 0, -3.0)), r, oracle.DRAG)
    np.testing.assert_allclose(d, [0, 0, P.c_z * k * 3.0], rtol=1e-13, atol=1e-20)
    # pitched by +90 deg the body z axis lies along world +x: a world-x velocity sees c_z
    d = _extra_fz(P, state(q=axis_angle((0, 1, 0), math.pi / 2), v=(2.0, 0, 0)), r, oracle.DRAG)
    np.testing.assert_allclose(d, [-P.c_z * k * 2.0, 0, 0], rtol=1e-12, atol=1e-18)


def test_drag_yaw_equivariance_and_dissipation():
    rng = np.random.default_rng(4)
    r = rng.uniform(0.8, 1.2, 4) * HOVER
    q0 = axis_angle(rng.normal(size=3), 0.7)
    v0 = rng.normal(size=3)
    d0 = _extra_fz(P, state(q=q0, v=v0), r, oracle.DRAG)
    assert d0 @ v0 < 0
    for psi in (0.3, 1.9, -2.5):
        qz = axis_angle((0, 0, 1), psi)
        Rz = np.array([[math.cos(psi), -math.sin(psi), 0], [math.sin(psi), math.cos(psi), 0], [0, 0, 1]])
        d = _extra_fz(P, state(q=qmul(qz, q0), v=Rz @ v0), r, oracle.DRAG)
        np.testing.assert_allclose(d, Rz @ d0, rtol=1e-12, atol=1e-20)


# ---------------------------------------------------------------- downwash
def _dw(xs, flags=oracle.DW, params=P):
    xs = np.asarray(xs, dtype=float)
    rpm = np.full((xs.shape[0], 4), HOVER)
    F1, _ = oracle.env_forces(params, xs, rpm, flags)
    F0, _ = oracle.env_forces(params, xs, rpm, 0)
    return F1 - F0


def test_downwash_coaxial_pair():
    # dxy = 0: the Gaussian factor is 1, the lower drone gets -C1 (r_p/(4 dz))^2, the upper nothing.
    d = _dw([state(p=(0, 0, 1.0)), state(p=(0, 0, 1.25))])
    assert d[1, 2] == 0.0 and np.all(d[:, :2] == 0)
    assert d[0, 2] == pytest.approx(-P.dw_c1 * (P.prop_radius / 1.0) ** 2, rel=1e-14)
    # about 4.6 times the weight at dz = 0.25 m
    assert -d[0, 2] / (P.mass * P.g) == pytest.approx(4.627, abs=1e-3)
    # inverse-square law in dz at zero lateral offset
    d2 = _dw([state(p=(0, 0, 1.0)), state(p=(0, 0, 1.5))])
    assert d[0, 2] / d2[0, 2] == pytest.approx(4.0, rel=1e-13)


def test_downwash_lateral_gaussian_width():
    dz = 0.9
    beta = abs(P.dw_c2 * dz + P.dw_c3)
    f0 = _dw([state(p=(0, 0, 0)), state(p=(0, 0, dz))])[0, 2]
    fb = _dw([state(p=(0, 0, 0)), state(p=(beta * 0.6, beta * 0.8, dz))])[0, 2]
    f2 = _dw([state(p=(0, 0, 0)), state(p=(2 * beta, 0, dz))])[0, 2]
    assert fb / f0 == pytest.approx(math.exp(-0.5), rel=1e-13)
    assert f2 / f0 == pytest.approx(math.exp(-2.0), rel=1e-13)


def test_downwash_equal_heights_and_cutoffs():
    assert np.all(_dw([state(p=(0, 0, 1)), state(p=(0.05, 0, 1))]) == 0)
    # beyond 10 m laterally nothing; inside, with a wide plume (large dz), something
    assert _dw([state(p=(0, 0, 0)), state(p=(10.5, 0, 50))])[0, 2] == 0
    assert _dw([state(p=(0, 0, 0)), state(p=(9.5, 0, 50))])[0, 2] < 0
    # beta = 0 at dz = -C3/C2: finite; full strength on the axis, none off it
    dz0 = -P.dw_c3 / P.dw_c2
    on = _dw([state(p=(0, 0, 0)), state(p=(0, 0, dz0))])[0, 2]
    off = _dw([state(p=(0, 0, 0)), state(p=(0.01, 0, dz0))])[0, 2]
    assert np.isfinite(on) and on < 0 and off == 0


def test_downwash_superposition_and_symmetry():
    low = state(p=(0.1, -0.2, 1.0))
    a = state(p=(0.25, -0.1, 1.3))
    b = state(p=(-0.1, 0.0, 1.1))
    d3 = _dw([low, a, b])
    da = _dw([low, a])
    db = _dw([low, b])
    assert d3[0, 2] == pytest.approx(da[0, 2] + db[0, 2], rel=1e-14)
    assert d3[2, 2] == pytest.approx(_dw([b, a])[0, 2], rel=1e-14)
    assert d3[1, 2] == 0
    # mirror x -> -x
    m = [s.copy() for s in (low, a, b)]
    for s in m:
        s[0] = -s[0]
    np.testing.assert_allclose(_dw(m)[:, 2], d3[:, 2], rtol=1e-14)


def test_substep_is_jacobi_permutation_invariant():
    rng = np.random.default_rng(5)
    N = 8
    xs = np.stack([state(p=rng.uniform([-0.3, -0.3, 0.8], [0.3, 0.3, 1.4]),
                         q=axis_angle(rng.normal(size=3), rng.uniform(0, 0.3)),
                         v=rng.normal(size=3) * 0.2, w=rng.normal(size=3)) for _ in range(N)])
    rpm = rng.uniform(0.9, 1.1, (N, 4)) * HOVER
    out = oracle.substep(P, xs, rpm, oracle.GND | oracle.DRAG | oracle.DW)
    perm = rng.permutation(N)
    outp = oracle.substep(P, xs[perm], rpm[perm], oracle.GND | oracle.DRAG | oracle.DW)
    np.testing.assert_allclose(outp, out[perm], rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- PID
def test_pid_at_waypoint_returns_hover_rpm():
    rpm, pe, ye, integ = oracle.pid(P, state(p=(0.4, -0.3, 1.2)), np.zeros(6), [0.4, -0.3, 1.2, 0.0])
    np.testing.assert_allclose(rpm, HOVER, rtol=1e-12)
    assert np.all(pe == 0) and ye == 0 and np.all(integ == 0)


def test_pid_torque_signs():
    def wrench(wp, x=None):
        rpm, _, _, _ = oracle.pid(P, state() if x is None else x, np.zeros(6), wp)
        return oracle.motor(P, rpm)

    T, tau = wrench([0, 0, 1.5, 0])  # straight up: pure thrust
    assert T > P.mass * P.g and np.all(np.abs(tau) < 1e-12 * T)
    _, tau = wrench([0.5, 0, 1, 0])   # +x: pitch up (theta* > 0)
    assert tau[1] > 0 and abs(tau[0]) < 1e-3 * tau[1]
    _, tau = wrench([0, 0.5, 1, 0])   # +y: roll negative
    assert tau[0] < 0 and abs(tau[1]) < 1e-3 * abs(tau[0])
    _, tau = wrench([0, 0, 1, 0.3])   # yaw target left: positive yaw torque
    assert tau[2] > 0
    # yaw error wraps: heading 3.0 rad to target -3.0 rad is +0.283 rad, not -6 rad
    _, _, ye, _ = oracle.pid(P, state(q=axis_angle((0, 0, 1), 3.0)), np.zeros(6), [0, 0, 1, -3.0])
    assert ye == pytest.approx(2 * math.pi - 6.0, abs=1e-12)


def test_pid_integrals_clamp():
    integ = np.zeros(6)
    for _ in range(500):
        _, _, _, integ = oracle.pid(P, state(), integ, [100.0, -100.0, 1.0, 0.0])
    assert integ[0] == 2.0 and integ[1] == -2.0 and integ[2] == 0.0
    assert np.all(np.abs(integ[3:]) <= 0.5)


def test_pid_closed_loop_reaches_waypoint():
    # Paper example pid_hover: the PID drives one drone to a waypoint and holds it.
    env_off = np.array([0, 1], dtype=np.int32)
    wp = np.array([0.3, -0.2, 1.0, 0.0])
    x, integ, a = oracle.control_steps(P, env_off, [0], [oracle.ACT_PID], state(p=(0, 0, 0.5))[None],
                                       np.zeros((1, 6)), np.zeros((1, 4)), np.tile(wp, (480, 1, 1)), 5)
    # settles within a few cm in 10 s (the small position K_i leaves a slow integral tail)
    assert np.linalg.norm(x[0, :3] - wp[:3]) < 0.03
    assert np.linalg.norm(x[0, 7:10]) < 0.01
    np.testing.assert_allclose(a[0], HOVER, rtol=0.01)


def test_stacked_pair_lower_drone_raises_thrust():
    # Paper Fig. downwash: under ground effect + drag + downwash the lower drone of a stacked
    # pair spins up against the upper drone's wake.
    env_off = np.array([0, 2], dtype=np.int32)
    xs = np.stack([state(p=(0, 0, 1.0)), state(p=(0, 0, 1.5))])
    wp = np.array([[0, 0, 1.0, 0], [0, 0, 1.5, 0]])
    x, integ, a = oracle.control_steps(P, env_off, [7], [oracle.ACT_PID], xs, np.zeros((2, 6)),
                                       np.zeros((2, 4)), np.tile(wp, (24, 1, 1)), 5)
    assert a[0].mean() > 1.1 * a[1].mean()
    # the upper drone feels no wake and holds its waypoint
    assert abs(x[1, 2] - 1.5) < 1e-3


def test_rpm_actions_are_clipped():
    env_off = np.array([0, 1], dtype=np.int32)
    _, _, a = oracle.control_steps(P, env_off, [0], [oracle.ACT_RPM], state()[None], np.zeros((1, 6)),
                                   np.zeros((1, 4)), np.array([[[-5.0, 1e9, 100.0, MAXRPM]]]), 1)
    np.testing.assert_array_equal(a[0], [0.0, MAXRPM, 100.0, MAXRPM])


# ---------------------------------------------------------------- observations
def test_kin_layout():
    x = np.arange(13, dtype=float) + 1
    x[3:7] = axis_angle((0.2, -0.4, 1.0), 0.5)
    a = np.array([101.0, 102, 103, 104])
    k = oracle.kin(x, a)
    np.testing.assert_array_equal(k[0:3], x[0:3])
    np.testing.assert_array_equal(k[3:7], x[3:7])
    np.testing.assert_allclose(k[7:10], oracle.rpy(x[3:7]))
    np.testing.assert_array_equal(k[10:13], x[7:10])
    np.testing.assert_array_equal(k[13:16], x[10:13])
    np.testing.assert_array_equal(k[16:20], a)


def _env(ps, vs=None):
    out = []
    for i, p in enumerate(ps):
        v = (0, 0, 0) if vs is None else vs[i]
        out.append(state(p=p, v=v))
    return np.stack(out)


def test_knn_collinear_and_padding():
    xs = _env([(0, 0, 1), (1, 0, 1), (3, 0, 1), (2, 0, 1), (8, 0, 1), (5, 0, 1)],
              [(0, 0, 0), (1, 0, 0), (3, 0, 0), (2, 0, 0), (8, 0, 0), (5, 0, 0)])
    idx, rel = oracle.knn(xs, 0, idx_base=100)
    np.testing.assert_array_equal(idx, [101, 103, 102, 105])
    np.testing.assert_allclose(rel.reshape(4, 6)[:, 0], [1, 2, 3, 5])
    np.testing.assert_allclose(rel.reshape(4, 6)[:, 3], [1, 2, 3, 5])
    idx, rel = oracle.knn(xs[:3], 2)
    np.testing.assert_array_equal(idx, [1, 0, -1, -1])
    assert np.all(rel[12:] == 0)
    idx, rel = oracle.knn(xs[:1], 0)
    np.testing.assert_array_equal(idx, [-1] * 4)


def test_knn_ties_take_lower_index():
    xs = _env([(0, 0, 1), (0, 1, 1), (1, 0, 1), (0, -1, 1), (-1, 0, 1), (0, 0, 2)])
    idx, _ = oracle.knn(xs, 0)
    np.testing.assert_array_equal(idx, [1, 2, 3, 4])
    idx, _ = oracle.knn(xs, 5)
    np.testing.assert_array_equal(idx, [0, 1, 2, 3])


def test_knn_brute_force_random():
    rng = np.random.default_rng(6)
    for N in (2, 5, 17, 64):
        xs = _env(rng.uniform(-1, 1, (N, 3)), rng.normal(size=(N, 3)))
        for j in range(N):
            idx, rel = oracle.knn(xs, j)
            d = np.linalg.norm(xs[:, :3] - xs[j, :3], axis=1)
            d[j] = np.inf
            order = np.argsort(d, kind="stable")[: min(4, N - 1)]
            np.testing.assert_array_equal(idx[: len(order)], order)
            for k, i in enumerate(order):
                np.testing.assert_allclose(rel[6 * k:6 * k + 3], xs[i, :3] - xs[j, :3])
                np.testing.assert_allclose(rel[6 * k + 3:6 * k + 6], xs[i, 7:10] - xs[j, 7:10])
