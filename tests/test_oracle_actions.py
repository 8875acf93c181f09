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
