"""Pins of the oracle's action types (Table "Action types"): normalized RPM, ONE_D_RPM,
VEL and ATTITUDE (CPU).

The normalized map is a reading (the paper names the mapping but does not print it): its
defining points are pinned. VEL and ATTITUDE are pinned by what the readings fix about the
closed loop, not by re-deriving their arithmetic: a zero command at hover gives the hover
RPMs; a body-frame velocity command at a yaw of 0.7 rad brings the world-frame velocity to
R_z(psi) v (no drag, so steady flight needs no tilt); a yaw-rate command brings the body
rate to it; an attitude command brings roll and pitch to it; neither touches the position
integrals it does not use.
"""
import numpy as np
import pytest

import oracle


def _x(p=(0.0, 0.0, 1.0), q=(1.0, 0.0, 0.0, 0.0), v=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0)):
    return np.array([*p, *q, *v, *w], np.float64)


def _yaw_quat(psi):
    return (np.cos(psi / 2), 0.0, 0.0, np.sin(psi / 2))


def _fly(P, x0, act_type, action, steps, flags=0):
    """Closed loop of one drone: `steps` control steps of 5 substeps with a fixed action."""
    x, integ, a = x0[None].copy(), np.zeros((1, 6)), np.zeros((1, 4))
    acts = np.repeat(np.asarray(action, np.float64)[None, None], steps, axis=0)
    x, integ, a = oracle.control_steps(P, np.array([0, 1], np.int32), np.array([flags], np.int32),
                                       np.array([act_type], np.int32), x, integ, a, acts, 5)
    return x[0], integ[0], a[0]


# ------------------------------------------------------------------ normalized RPM
def test_normalized_map_defining_points():
    for P in (oracle.cf2x(), oracle.race()):
        h, m = oracle.hover_rpm(P), oracle.max_rpm(P)
        assert oracle.normalized_rpm(P, -1.0) == 0.0
        assert oracle.normalized_rpm(P, 0.0) == pytest.approx(h, rel=1e-15)
        assert oracle.normalized_rpm(P, 1.0) == pytest.approx(m, rel=1e-15)
        assert oracle.normalized_rpm(P, -0.5) == pytest.approx(0.5 * h, rel=1e-15)
        assert oracle.normalized_rpm(P, 0.5) == pytest.approx(0.5 * (h + m), rel=1e-15)
        assert oracle.normalized_rpm(P, -3.0) == 0.0 and oracle.normalized_rpm(P, 7.0) == pytest.approx(m)
        a = np.linspace(-1, 1, 41)
        r = np.array([oracle.normalized_rpm(P, t) for t in a])
        assert np.all(np.diff(r) > 0)


def test_normalized_and_one_d_actions_through_control_steps():
    """RPM_NORM and ONE_D_RPM control steps equal RPM control steps with the mapped speeds."""
    P = oracle.cf2x()
    x0 = _x(p=(0.1, 0.2, 0.8))
    a_norm = np.array([-0.2, 0.1, 0.35, -0.6])
    mapped = np.array([oracle.normalized_rpm(P, t) for t in a_norm])
    xa, _, ra = _fly(P, x0, oracle.ACT_RPM_NORM, a_norm, 3, flags=oracle.GND | oracle.DRAG)
    xb, _, rb = _fly(P, x0, oracle.ACT_RPM, mapped, 3, flags=oracle.GND | oracle.DRAG)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ra, rb)
    xc, _, rc = _fly(P, x0, oracle.ACT_ONE_D_RPM, [0.3, -0.9, 0.9, 0.0], 3)
    xd, _, rd = _fly(P, x0, oracle.ACT_RPM, np.full(4, oracle.normalized_rpm(P, 0.3)), 3)
    np.testing.assert_array_equal(xc, xd)
    np.testing.assert_array_equal(rc, rd)


# ------------------------------------------------------------------ VEL
@pytest.mark.parametrize("model", ["cf2x", "cf2p"])
def test_vel_zero_command_at_hover_gives_hover_rpm(model):
    P = getattr(oracle, model)()
    rpm, integ = oracle.action_to_rpm(P, oracle.ACT_VEL, _x(q=_yaw_quat(0.4)), np.zeros(6), [0, 0, 0, 0])
    np.testing.assert_allclose(rpm, oracle.hover_rpm(P), rtol=1e-12)
    np.testing.assert_array_equal(integ, 0.0)


def test_vel_tracks_the_body_frame_velocity():
    """Yaw 0.7 rad, no drag: the velocity loop (Kd) drives v to R_z(psi) v_body; the
    position integrals stay zero (e_p = 0)."""
    P = oracle.cf2x()
    psi = 0.7
    vb = np.array([0.6, -0.3, 0.2])
    x, integ, _ = _fly(P, _x(q=_yaw_quat(psi)), oracle.ACT_VEL, [*vb, 0.0], 48 * 6)
    c, s = np.cos(psi), np.sin(psi)
    v_world = np.array([c * vb[0] - s * vb[1], s * vb[0] + c * vb[1], vb[2]])
    np.testing.assert_allclose(x[7:10], v_world, atol=2e-3)
    np.testing.assert_array_equal(integ[0:3], 0.0)
    assert abs(oracle.rpy(x[3:7])[2] - psi) < 2e-3


def test_vel_yaw_rate_command():
    P = oracle.cf2x()
    x, _, _ = _fly(P, _x(), oracle.ACT_VEL, [0.0, 0.0, 0.0, 0.8], 48 * 3)
    assert x[12] == pytest.approx(0.8, abs=2e-3)
    assert np.linalg.norm(x[7:10]) < 2e-2


# ------------------------------------------------------------------ ATTITUDE
def test_attitude_hover_command_gives_hover_rpm():
    P = oracle.cf2x()
    rpm, integ = oracle.action_to_rpm(P, oracle.ACT_ATTITUDE, _x(), np.zeros(6), [P.mass * P.g, 0, 0, 0])
    np.testing.assert_allclose(rpm, oracle.hover_rpm(P), rtol=1e-12)
    np.testing.assert_array_equal(integ, 0.0)


@pytest.mark.parametrize("model", ["cf2x", "cf2p", "race"])
def test_attitude_command_reaches_roll_and_pitch(model):
    P = getattr(oracle, model)()
    phi, theta = 0.15, -0.1
    T = P.mass * P.g / (np.cos(phi) * np.cos(theta))
    x, integ, _ = _fly(P, _x(p=(0, 0, 5.0)), oracle.ACT_ATTITUDE, [T, phi, theta, 0.0], 48 * 2)
    rpy = oracle.rpy(x[3:7])
    assert rpy[0] == pytest.approx(phi, abs=2e-3)
    assert rpy[1] == pytest.approx(theta, abs=2e-3)
    np.testing.assert_array_equal(integ[0:3], 0.0)


@pytest.mark.parametrize("model", ["cf2x", "race"])
def test_attitude_yaw_rate_command(model):
    """Level, hover thrust, yaw rate 0.5 rad/s: the body rate about z settles at 0.5. (At a
    tilt the same command leaves a roll/pitch offset: turning needs body roll and pitch
    rates, which the rate term with target [0, 0, r] opposes.)"""
    P = getattr(oracle, model)()
    x, _, _ = _fly(P, _x(p=(0, 0, 5.0)), oracle.ACT_ATTITUDE, [P.mass * P.g, 0.0, 0.0, 0.5], 48 * 3)
    assert x[12] == pytest.approx(0.5, abs=2e-3)
    np.testing.assert_allclose(oracle.rpy(x[3:7])[0:2], 0.0, atol=1e-6)


# ------------------------------------------------------------------ DSL controller
def test_dsl_setpoint_limiter():
    """The setpoint starts at the drone (NaN = not set), moves 2.0 m/s x dt_ctrl along the
    straight line to a far waypoint, lands exactly on a near one, and turns the yaw by at
    most pi x dt_ctrl the short way across +-pi."""
    P = oracle.controller_dsl(oracle.cf2x())
    x = _x(p=(0.3, -0.2, 1.1), q=_yaw_quat(0.25))
    step = 2.0 * P.dt_ctrl
    sp = oracle.dsl_setpoint(P, x, [0.3, -0.2, 1.1, 0.25], oracle.new_setpoints(1)[0])
    np.testing.assert_allclose(sp, [0.3, -0.2, 1.1, 0.25], atol=1e-15)
    far = np.array([3.3, 3.8, 1.1 + 12.0 / 5 * 0, 0.25])
    d = far[0:3] - sp[0:3]
    sp2 = oracle.dsl_setpoint(P, x, far, sp)
    np.testing.assert_allclose(sp2[0:3], sp[0:3] + step * d / np.linalg.norm(d), rtol=0, atol=1e-15)
    assert sp2[3] == pytest.approx(0.25, abs=1e-15)
    near = sp2 + np.array([0.5 * step, 0.0, 0.0, 0.0])
    np.testing.assert_allclose(oracle.dsl_setpoint(P, x, near, sp2), near, atol=1e-15)
    # yaw: setpoint at 3.1 rad, waypoint at -3.1 rad: the short way is +0.083 rad through pi
    sp3 = np.array([0.0, 0.0, 1.0, 3.1])
    y = oracle.dsl_setpoint(P, x, [0.0, 0.0, 1.0, -3.1], sp3)[3]
    expected = 3.1 + np.pi * P.dt_ctrl
    expected -= 2 * np.pi if expected >= np.pi else 0.0
    assert y == pytest.approx(expected, abs=1e-14)
    y = oracle.dsl_setpoint(P, x, [0.0, 0.0, 1.0, 2.0], np.array([0.0, 0.0, 1.0, 3.1]))[3]
    assert y == pytest.approx(3.1 - np.pi * P.dt_ctrl, abs=1e-14)


def test_feed_forward_enters_the_position_loop():
    """At its waypoint with a feed-forward acceleration (1, 0, 0) m/s^2, the PID commands
    what an ATTITUDE action with T = m sqrt(1 + g^2), pitch 1/g (small-angle target of
    a* = (1, 0, g)) commands; (0, 0, 1) scales the hover speeds by sqrt((g + 1)/g)."""
    for P in (oracle.cf2x(), oracle.controller_dsl(oracle.cf2x())):
        x = _x(p=(0.2, 0.1, 1.0))
        wp = [0.2, 0.1, 1.0, 0.0]
        sp = oracle.new_setpoints(1)[0]
        rpm, _, _, _, _ = oracle.pid_ff(P, x, np.zeros(6), wp, a_ff=[1.0, 0.0, 0.0], sp=sp)
        ref, _ = oracle.action_to_rpm(P, oracle.ACT_ATTITUDE, x, np.zeros(6),
                                      [P.mass * np.sqrt(1.0 + P.g ** 2), 0.0, 1.0 / P.g, 0.0])
        np.testing.assert_allclose(rpm, ref, rtol=1e-13)
        rpm, _, _, _, _ = oracle.pid_ff(P, x, np.zeros(6), wp, a_ff=[0.0, 0.0, 1.0], sp=sp)
        np.testing.assert_allclose(rpm, oracle.hover_rpm(P) * np.sqrt((P.g + 1.0) / P.g), rtol=1e-13)


def test_dsl_closed_loop_is_rate_limited_and_converges():
    """Towards a waypoint 6 m away (a 3 s setpoint ramp) the DSL drone speeds up to about
    its 2.0 m/s setpoint rate, never much beyond it, and settles on the waypoint."""
    P = oracle.controller_dsl(oracle.cf2x())
    wp = np.array([6.0, 0.0, 1.0, 0.0])
    x, integ, a = _x(p=(0.0, 0.0, 1.0))[None], np.zeros((1, 6)), np.zeros((1, 4))
    sp = oracle.new_setpoints(1)
    speeds = []
    for _ in range(48 * 7):
        x, integ, a = oracle.control_steps(P, np.array([0, 1], np.int32), np.array([0], np.int32),
                                           np.array([oracle.ACT_PID], np.int32), x, integ, a, wp[None, None], 5,
                                           setpoint=sp)
        speeds.append(np.linalg.norm(x[0, 7:10]))
    assert max(speeds) < 2.3, max(speeds)
    assert max(speeds) > 1.8  # it does fly at about the limit
    assert np.linalg.norm(x[0, 0:3] - wp[0:3]) < 0.05  # after a ~5 cm overshoot
    np.testing.assert_allclose(sp[0], wp, atol=1e-12)


def test_dsl_setpoints_carry_across_calls():
    P = oracle.controller_dsl(oracle.cf2x())
    x0 = np.stack([_x(p=(0.1 * j, 0.0, 1.0)) for j in range(3)])
    wp = np.array([[2.0, 1.0, 1.5, 0.5]] * 3)
    args = (np.array([0, 3], np.int32), np.array([0], np.int32), np.array([oracle.ACT_PID], np.int32))
    sa = oracle.new_setpoints(3)
    xa, ia, aa = oracle.control_steps(P, *args, x0, np.zeros((3, 6)), np.zeros((3, 4)),
                                      np.repeat(wp[None], 4, axis=0), 5, setpoint=sa)
    sb = oracle.new_setpoints(3)
    xb, ib, ab = x0, np.zeros((3, 6)), np.zeros((3, 4))
    for _ in range(4):
        xb, ib, ab = oracle.control_steps(P, *args, xb, ib, ab, wp[None], 5, setpoint=sb)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(sa, sb)
    with pytest.raises(ValueError):
        oracle.control_steps(P, *args, x0, np.zeros((3, 6)), np.zeros((3, 4)), wp[None], 5)
