"""Pins of the oracle's model and integrator variants (CPU): the RK4 substep, the +
rotor layout (CF2P) and the RACE constants.

Nothing here re-derives the oracle's code: RK4 is pinned by exact solutions (free fall,
hover, principal-axis spin), by its measured convergence order (error x16 smaller per
halving of dt, against Euler's x2) on tumbling single drones and on a stacked pair whose
downwash couples the stages, and by angular-momentum conservation; the + layout by its
torque special cases and its allocation round trip; RACE by the printed table and by the
controller reaching a waypoint with the gains read for it.
"""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _rk4(p):
    q = oracle.Params()
    ctypes_copy(p, q)
    q.integrator = oracle.RK4
    return q


def ctypes_copy(src, dst):
    import ctypes
    ctypes.memmove(ctypes.byref(dst), ctypes.byref(src), ctypes.sizeof(src))


def _level(p=(0.0, 0.0, 1.0), v=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0), q=(1.0, 0.0, 0.0, 0.0)):
    return np.array([[*p, *q, *v, *w]], np.float64)


def _run(P, x, rpm, flags, dt, n, rk4=True):
    for _ in range(n):
        x = oracle.substep_rk4(P, x, rpm, flags, dt) if rk4 else oracle.substep(P, x, rpm, flags, dt)
    return x


# ------------------------------------------------------------------ RK4 exact cases
def test_rk4_free_fall_is_exact():
    """With the rotors off, p'' = -g: RK4 integrates the quadratic exactly (to rounding)."""
    P = oracle.cf2x()
    x0 = _level(p=(0.3, -0.2, 5.0), v=(1.0, -0.5, 2.0))
    dt, n = P.dt_sim, 40
    x = _run(P, x0, np.zeros((1, 4)), 0, dt, n)
    t = dt * n
    np.testing.assert_allclose(x[0, 0:3], x0[0, 0:3] + x0[0, 7:10] * t - np.array([0, 0, 0.5 * P.g * t * t]),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(x[0, 7:10], x0[0, 7:10] - np.array([0, 0, P.g * t]), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(x[0, 3:7], x0[0, 3:7])


def test_rk4_hover_holds():
    P = oracle.cf2x()
    h = oracle.hover_rpm(P)
    x = _run(P, _level(), np.full((1, 4), h), 0, P.dt_sim, 240)
    np.testing.assert_allclose(x[0, 0:3], [0, 0, 1], atol=1e-11)
    np.testing.assert_allclose(x[0, 7:13], 0, atol=1e-10)


def test_rk4_principal_axis_spin():
    """Torque-free spin about z with Jxx = Jyy keeps w constant; q(t) = q0 (x) [cos(wt/2), 0, 0,
    sin(wt/2)]. RK4's quaternion error is O((w dt)^5) per step."""
    P = oracle.cf2x()
    wz = 3.0
    dt, n = P.dt_sim, 120
    x = _run(P, _level(w=(0.0, 0.0, wz)), np.zeros((1, 4)), 0, dt, n)
    t = dt * n
    np.testing.assert_allclose(x[0, 10:13], [0, 0, wz], atol=1e-13)
    np.testing.assert_allclose(x[0, 3:7], [np.cos(wz * t / 2), 0, 0, np.sin(wz * t / 2)], atol=1e-11)


# ------------------------------------------------------------------ convergence order
def _tumbling(seed, N=1):
    rng = np.random.default_rng(seed)
    x = np.zeros((N, 13))
    for j in range(N):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        x[j] = [*rng.uniform(-0.5, 0.5, 2), 0.15 + 0.3 * j, *q, *rng.uniform(-1, 1, 3), *rng.uniform(-4, 4, 3)]
    return x


def _order(P, x0, rpm, flags, rk4, T=12 / 240.0, steps=(12, 24, 48)):
    """Errors of x(T) after n substeps of T/n against a run with 16x the finest count."""
    ref = _run(P, x0, rpm, flags, T / (16 * steps[-1]), 16 * steps[-1], rk4=True)
    errs = []
    for n in steps:
        x = _run(P, x0, rpm, flags, T / n, n, rk4=rk4)
        errs.append(np.max(np.abs(x - ref)))
    return np.array(errs)


@pytest.mark.parametrize("flags", [0, oracle.GND | oracle.DRAG])
def test_rk4_is_fourth_order_and_euler_first(flags):
    P = oracle.cf2x()
    x0 = _tumbling(3)
    rpm = np.array([[14000.0, 15500.0, 13000.0, 16000.0]])
    e4 = _order(P, x0, rpm, flags, rk4=True)
    r4 = e4[:-1] / e4[1:]
    assert np.all((r4 > 12) & (r4 < 21)), r4
    e1 = _order(P, x0, rpm, flags, rk4=False)
    r1 = e1[:-1] / e1[1:]
    assert np.all((r1 > 1.6) & (r1 < 2.5)), r1


def test_rk4_order_holds_with_downwash_coupling():
    """A stacked pair (dz = 0.3 m) under downwash: the stages must evaluate every drone's
    force at that stage's positions, else the order collapses."""
    P = oracle.cf2x()
    x0 = _tumbling(5, N=2)
    x0[:, 10:13] *= 0.1
    x0[1, 0:2] = x0[0, 0:2] + 0.01
    x0[1, 7:10] = [0.0, 0.0, -1.5]  # the upper drone sinks towards the lower one
    rpm = np.full((2, 4), 14500.0)
    e4 = _order(P, x0, rpm, oracle.DW | oracle.GND | oracle.DRAG, rk4=True)
    r4 = e4[:-1] / e4[1:]
    assert np.all((r4 > 12) & (r4 < 21)), r4


def test_rk4_conserves_angular_momentum_far_better_than_euler():
    """Torque-free tumbling (rotors off): |J w| is constant; RK4 keeps it to O(dt^4)."""
    P = oracle.cf2x()
    x0 = _tumbling(7)
    x0[0, 10:13] = [5.0, -3.0, 2.0]
    J = np.array([P.Jxx, P.Jyy, P.Jzz])
    L0 = np.linalg.norm(J * x0[0, 10:13])
    x4 = _run(P, x0, np.zeros((1, 4)), 0, P.dt_sim, 240, rk4=True)
    x1 = _run(P, x0, np.zeros((1, 4)), 0, P.dt_sim, 240, rk4=False)
    d4 = abs(np.linalg.norm(J * x4[0, 10:13]) - L0) / L0
    d1 = abs(np.linalg.norm(J * x1[0, 10:13]) - L0) / L0
    assert d4 < 1e-8 and d1 > 1e3 * d4, (d4, d1)


def test_rk4_through_control_steps_matches_direct_substeps():
    """orc_control_steps with integrator = RK4 applies orc_substep_rk4 n_sub times."""
    P = _rk4(oracle.cf2x())
    x0 = _tumbling(9, N=3)
    rpm = np.full((3, 4), 14600.0)
    env_off = np.array([0, 3], np.int32)
    xa, _, _ = oracle.control_steps(P, env_off, np.array([7], np.int32), np.array([oracle.ACT_RPM], np.int32),
                                    x0, np.zeros((3, 6)), np.zeros((3, 4)), rpm[None], 5)
    xb = _run(P, x0, rpm, 7, P.dt_sim, 5)
    np.testing.assert_array_equal(xa, xb)


# ------------------------------------------------------------------ + rotor layout
def test_plus_layout_torques():
    """CF2P: rotors at L (+x, +y, -x, -y): one rotor alone gives the torque of its lever
    arm, and the yaw signs are those of the X layout."""
    P = oracle.cf2p()
    n = 15000.0
    F = P.kf * n * n
    cases = {0: (0.0, -P.arm * F, -P.km * n * n), 1: (P.arm * F, 0.0, P.km * n * n),
             2: (0.0, P.arm * F, -P.km * n * n), 3: (-P.arm * F, 0.0, P.km * n * n)}
    for i, (tx, ty, tz) in cases.items():
        rpm = np.zeros(4)
        rpm[i] = n
        T, tau = oracle.motor(P, rpm)
        assert T == pytest.approx(F, rel=1e-15)
        np.testing.assert_allclose(tau, [tx, ty, tz], rtol=1e-14, atol=1e-20)


def test_plus_layout_allocation_round_trip():
    P = oracle.cf2p()
    M = oracle.allocation_matrix(P)
    rng = np.random.default_rng(11)
    for _ in range(5):
        f = rng.uniform(0.01, 0.08, 4)
        rpm = np.sqrt(f / P.kf)
        T, tau = oracle.motor(P, rpm)
        np.testing.assert_allclose(M @ f, [T, *tau], rtol=1e-12)


@pytest.mark.parametrize("model", ["cf2p", "race"])
def test_pid_at_waypoint_returns_hover_rpm(model):
    P = getattr(oracle, model)()
    x = _level(p=(0.4, -0.3, 1.2))[0]
    rpm, _, _, _ = oracle.pid(P, x, np.zeros(6), np.array([0.4, -0.3, 1.2, 0.0]))
    np.testing.assert_allclose(rpm, oracle.hover_rpm(P), rtol=1e-12)


def _closed_loop(P, steps=240):
    x = _level(p=(0.0, 0.0, 1.0))
    wp = np.array([[0.5, -0.3, 1.4, 0.7]])
    xo, _, _ = oracle.control_steps(P, np.array([0, 1], np.int32), np.array([0], np.int32),
                                    np.array([oracle.ACT_PID], np.int32), x, np.zeros((1, 6)), np.zeros((1, 4)),
                                    np.repeat(wp[None], steps, axis=0), 5)
    return xo[0], wp[0]


def test_closed_loop_of_the_other_models():
    """With the PID in the loop (5 s towards a waypoint 0.7 m away, yaw 0.7 rad): CF2P
    follows the CF2X trajectory to rounding (its allocation inverts the + mixing exactly),
    RACE with its inertia-scaled attitude gains follows it closely, and all reach the
    waypoint."""
    x_x, wp = _closed_loop(oracle.cf2x())
    x_p, _ = _closed_loop(oracle.cf2p())
    x_r, _ = _closed_loop(oracle.race())
    np.testing.assert_allclose(x_p, x_x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(x_r, x_x, rtol=0, atol=1e-3)
    for x in (x_x, x_p, x_r):
        assert np.linalg.norm(x[0:3] - wp[0:3]) < 0.05
        assert np.linalg.norm(x[7:10]) < 0.1


def test_race_constants_match_the_printed_table():
    g = json.load(open(os.path.join(HERE, "golden", "race_paper_constants.json")))
    o = oracle.race().to_dict()
    for k, v in g.items():
        if not k.startswith("_"):
            np.testing.assert_allclose(o[k], v["value"], rtol=1e-15, err_msg=k)
    P = oracle.race()
    assert oracle.hover_rpm(P) == pytest.approx(np.sqrt(P.mass * P.g / (4 * P.kf)), rel=1e-15)
    assert 4 * P.kf * oracle.max_rpm(P) ** 2 == pytest.approx(P.thrust2weight * P.mass * P.g, rel=1e-14)


# ------------------------------------------------------------------ per-rotor ground-effect heights
def _gnd_rotor(P):
    P.gnd_heights = oracle.GND_ROTOR
    return P


@pytest.mark.parametrize("model", ["cf2x", "cf2p", "race"])
def test_rotor_positions_reproduce_the_torque_equations(model):
    """tau = sum_i r_i x (0, 0, F_i) with the rotor positions equals orc_motor's roll and
    pitch torques (Section 3.1.2) for random rotor speeds."""
    P = getattr(oracle, model)()
    r = np.array([oracle.rotor_position(P, i) for i in range(4)])
    assert np.all(r[:, 2] == 0)
    np.testing.assert_allclose(np.hypot(r[:, 0], r[:, 1]), P.arm, rtol=1e-15)
    rng = np.random.default_rng(21)
    for _ in range(5):
        rpm = rng.uniform(5000, 20000, 4)
        F = P.kf * rpm ** 2
        _, tau = oracle.motor(P, rpm)
        tau_geo = np.cross(r, np.stack([np.zeros(4), np.zeros(4), F], axis=1)).sum(axis=0)
        np.testing.assert_allclose(tau[:2], tau_geo[:2], rtol=1e-13, atol=1e-22)


@pytest.mark.parametrize("model", ["cf2x", "cf2p"])
def test_per_rotor_ground_effect_of_a_level_drone_is_the_printed_one(model):
    """Level: every rotor sits at p_z, so the variant equals Eq. ground at the CoM height,
    also below h_clip."""
    Pc = getattr(oracle, model)()
    Pr = _gnd_rotor(getattr(oracle, model)())
    rng = np.random.default_rng(22)
    for z in (0.005, Pc.h_clip, 0.03, 0.2, 1.5):
        x = _level(p=(0.1, -0.2, z), v=(0.3, 0.1, -0.2))
        rpm = rng.uniform(10000, 20000, (1, 4))
        Fc, _ = oracle.env_forces(Pc, x, rpm, oracle.GND)
        Fr, _ = oracle.env_forces(Pr, x, rpm, oracle.GND)
        np.testing.assert_allclose(Fr, Fc, rtol=1e-14, atol=0)


def _axis_quat(axis, angle):
    q = np.zeros(4)
    q[0] = np.cos(angle / 2)
    q[1 + axis] = np.sin(angle / 2)
    return q


@pytest.mark.parametrize("model, axis, rotor, offset", [
    # X layout, rotor 0 at (l, l): rolled by phi about body x its height is z + l sin(phi),
    # pitched by theta about body y it is z - l sin(theta) (l = L/sqrt2)
    ("cf2x", 0, 0, lambda P, a: P.arm / np.sqrt(2) * np.sin(a)),
    ("cf2x", 1, 0, lambda P, a: -P.arm / np.sqrt(2) * np.sin(a)),
    ("cf2x", 0, 2, lambda P, a: -P.arm / np.sqrt(2) * np.sin(a)),
    # + layout: rotor 1 on +y rises with roll, rotor 0 on +x sinks with pitch, rotor 0 does
    # not move under roll
    ("cf2p", 0, 1, lambda P, a: P.arm * np.sin(a)),
    ("cf2p", 1, 0, lambda P, a: -P.arm * np.sin(a)),
    ("cf2p", 0, 0, lambda P, a: 0.0),
])
def test_per_rotor_ground_effect_of_one_rotor_on_a_tilted_drone(model, axis, rotor, offset):
    """One rotor spinning on a drone tilted about a body axis: the increment is Eq. ground
    for that rotor at the height its lever arm gives it (hand geometry), thrust along the
    tilted body z axis."""
    P = _gnd_rotor(getattr(oracle, model)())
    z, ang, n = 0.08, 0.4, 16000.0
    x = _level(p=(0.0, 0.0, z), q=_axis_quat(axis, ang))
    rpm = np.zeros((1, 4))
    rpm[0, rotor] = n
    F, _ = oracle.env_forces(P, x, rpm, oracle.GND)
    f = P.kf * n * n
    h = z + offset(P, ang)
    expected = f * np.cos(ang) - P.mass * P.g + P.c_gnd * f * (P.prop_radius / (4 * h)) ** 2
    assert F[0, 2] == pytest.approx(expected, rel=1e-13)


def test_per_rotor_ground_effect_clips_each_rotor():
    """A rotor lowered below h_clip is clipped on its own: at p_z = h_clip and roll phi, rotor 2
    (lowered) sees h_clip, rotor 0 (raised) h_clip + l sin(phi)."""
    P = _gnd_rotor(oracle.cf2x())
    ang, n = 0.3, 15000.0
    x = _level(p=(0.0, 0.0, P.h_clip), q=_axis_quat(0, ang))
    f = P.kf * n * n
    for rotor, h in ((2, P.h_clip), (0, P.h_clip + P.arm / np.sqrt(2) * np.sin(ang))):
        rpm = np.zeros((1, 4))
        rpm[0, rotor] = n
        F, _ = oracle.env_forces(P, x, rpm, oracle.GND)
        gnd = F[0, 2] - (f * np.cos(ang) - P.mass * P.g)
        assert gnd == pytest.approx(P.c_gnd * f * (P.prop_radius / (4 * h)) ** 2, rel=1e-12)


def test_per_rotor_ground_effect_symmetry_and_convexity():
    """Equal rotor speeds: rolling by +phi or -phi gives the same force (the rotor pairs swap
    heights), and since 1/h^2 is convex the per-rotor increment exceeds the CoM one for a
    tilted drone whose rotors all stay above h_clip (Jensen)."""
    Pc, Pr = oracle.cf2x(), _gnd_rotor(oracle.cf2x())
    rpm = np.full((1, 4), 15000.0)
    for axis in (0, 1):
        xp = _level(p=(0.2, 0.1, 0.06), q=_axis_quat(axis, 0.35))
        xm = _level(p=(0.2, 0.1, 0.06), q=_axis_quat(axis, -0.35))
        Fp, _ = oracle.env_forces(Pr, xp, rpm, oracle.GND)
        Fm, _ = oracle.env_forces(Pr, xm, rpm, oracle.GND)
        np.testing.assert_allclose(Fp[0, 2], Fm[0, 2], rtol=1e-14)
        Fc, _ = oracle.env_forces(Pc, xp, rpm, oracle.GND)
        assert Fp[0, 2] > Fc[0, 2] + 1e-6
