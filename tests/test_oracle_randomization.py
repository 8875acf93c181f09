"""Pins of the oracle's domain randomization and wind (CPU).

The factors, the actuator effects and the wind models are pinned by what they fix in
special cases worked out by hand: neutral rows change nothing (bit for bit); at hover a
mass, gravity or thrust factor gives the exact constant acceleration it implies; inertia
and arm factors scale a single rotor's roll acceleration by their ratio; motor bias and
saturation equal pre-scaled RPM actions; the motor lag follows its geometric closed form;
latency replays the actions shifted by the delay; a steady wind pushes with
k |v_rel| v_rel and the sinusoid with its closed form; the Dryden process has the stationary
variance and lag-one correlation of its recursion and Gaussian innovations; gusts follow
the sin(pi s) envelope and trigger at the set rate in directions uniform on the sphere; the
counter-based uniforms equal those of the input generator (two implementations of the same
published SplitMix64 rounds).
"""
import numpy as np
import pytest

import oracle
from paper_2606_08039_gb300 import workloads as wl

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)


def _level(z=5.0, v=(0.0, 0.0, 0.0)):
    return np.array([[0.0, 0.0, z, 1.0, 0.0, 0.0, 0.0, *v, 0.0, 0.0, 0.0]])


def _run(x0, actions, dr=None, flags=0, act=oracle.ACT_RPM, P=P):
    """One drone (or a batch of single-drone envs) over actions [K, n, 4]."""
    n = x0.shape[0]
    env_off = np.arange(n + 1, dtype=np.int32)
    x, integ, a = oracle.control_steps(P, env_off, np.full(n, flags, np.int32), np.full(n, act, np.int32), x0,
                                       np.zeros((n, 6)), np.zeros((n, 4)), np.asarray(actions, np.float64), 5, dr=dr)
    return x, a


def _dr(n=1, depth=1, seed=0, **set_):
    r = oracle.Randomization(n, n, depth, seed)
    for k, v in set_.items():
        idx = getattr(oracle, "DR_" + k.upper())
        r.env_dr[:, idx:idx + np.size(v)] = v
    return r


def test_neutral_rows_change_nothing():
    sw = wl.uneven(3, n_envs=60)
    x0 = np.concatenate([sw.p, sw.q, sw.v, sw.w], 1).astype(np.float64)
    acts = np.stack([wl.mixed_actions(sw, 4, k, HOVER) for k in range(3)]).astype(np.float64)
    env_off = np.concatenate([[0], np.cumsum(sw.drones_per_env)]).astype(np.int32)
    args = (env_off, sw.flags.astype(np.int32), sw.act_type.astype(np.int32))
    z6, z4 = np.zeros((sw.n, 6)), np.zeros((sw.n, 4))
    xa, ia, aa = oracle.control_steps(P, *args, x0, z6, z4, acts, 5)
    r = oracle.Randomization(sw.n_envs, sw.n, depth=3, seed=9)
    xb, ib, ab = oracle.control_steps(P, *args, x0, z6, z4, acts, 5, dr=r)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(aa, ab)
    np.testing.assert_array_equal(r.wind[:, 7], 3)  # the wind steps advance even when idle


@pytest.mark.parametrize("factor, expected", [
    ("mass", lambda f: P.g * (1.0 / f - 1.0)),   # hover thrust m g on f m
    ("g", lambda f: -P.g * (f - 1.0)),
    ("kf", lambda f: P.g * (f - 1.0))])
def test_body_factors_at_hover(factor, expected):
    f = 1.2 if factor != "g" else 1.02
    x, _ = _run(_level(), np.full((1, 1, 4), HOVER), dr=_dr(**{factor: f}))
    assert x[0, 9] == pytest.approx(expected(f) * P.dt_ctrl, rel=1e-12)
    np.testing.assert_allclose(x[0, 7:9], 0.0, atol=1e-15)


def test_inertia_and_arm_factors_scale_the_roll_acceleration():
    rpm = np.array([[[12000.0, 0.0, 0.0, 0.0]]])
    x1, _ = _run(_level(), rpm, dr=_dr())
    x2, _ = _run(_level(), rpm, dr=_dr(j=[1.5, 1.0, 1.0], arm=1.02))
    w1, w2 = x1[0, 10], x2[0, 10]
    assert abs(w1) > 1.0
    assert w2 / w1 == pytest.approx(1.02 / 1.5, rel=1e-5)  # gyroscopic coupling enters at O(w^2 dt)
    # at rest (no gyroscopic term) the ratio of the instantaneous accelerations is exact
    row = oracle.neutral_dr(1)[0]
    row[oracle.DR_J], row[oracle.DR_ARM] = 1.5, 1.02
    d1 = oracle.env_deriv(P, _level(), rpm[0], 0)
    d2 = oracle.env_deriv(oracle.params_randomized(P, row), _level(), rpm[0], 0)
    assert d2[0, 10] / d1[0, 10] == pytest.approx(1.02 / 1.5, rel=1e-14)
    assert d2[0, 11] / d1[0, 11] == pytest.approx(1.02, rel=1e-14)  # pitch: arm only, Jyy unscaled


def test_drag_factor_scales_the_drag_force():
    x = _level(v=(1.5, 0.0, 0.0))[0]
    rpm = np.full((1, 4), HOVER)
    F0, _ = oracle.env_forces(P, x[None], rpm, oracle.DRAG)
    Fn, _ = oracle.env_forces(P, x[None], rpm, 0)
    row = oracle.neutral_dr(1)[0]
    row[oracle.DR_CXY] = 1.3
    F1, _ = oracle.env_forces(oracle.params_randomized(P, row), x[None], rpm, oracle.DRAG)
    assert (F1 - Fn)[0, 0] == pytest.approx(1.3 * (F0 - Fn)[0, 0], rel=1e-12)
    assert abs((F0 - Fn)[0, 0]) > 0


def test_motor_bias_and_saturation():
    bias = np.array([1.05, 1.0, 0.97, 1.02])
    a = np.array([[[14000.0, 15000.0, 13500.0, 14500.0]]])
    xa, _ = _run(_level(), a, dr=_dr(bias=bias), flags=oracle.DRAG)
    xb, _ = _run(_level(), a * bias, flags=oracle.DRAG)
    np.testing.assert_array_equal(xa, xb)
    mx = oracle.max_rpm(P)
    xa, aa = _run(_level(), np.full((1, 1, 4), mx), dr=_dr(maxrpm=0.95))
    xb, _ = _run(_level(), np.full((1, 1, 4), 0.95 * mx))
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_allclose(aa, mx)  # a_prev records the action's RPMs


def test_motor_lag_closed_form():
    """Motors at hover speed commanded to 1.1 x hover with tau = 30 ms: before substep s the
    speed is c + (n0 - c) e^(s+1), e = exp(-dt/tau); level and without effects the climb
    rate after one control step is the sum of the substeps' accelerations times dt."""
    tau, c, n0 = 0.03, 1.1 * HOVER, HOVER
    r = _dr(tau=tau)
    r.motor[:] = n0
    x, _ = _run(_level(), np.full((1, 1, 4), c), dr=r)
    e = np.exp(-P.dt_sim / tau)
    n = c + (n0 - c) * e ** np.arange(1, 6)
    vz = np.sum(P.dt_sim * (4 * P.kf * n ** 2 / P.mass - P.g))
    assert x[0, 9] == pytest.approx(vz, rel=1e-12)
    np.testing.assert_allclose(r.motor[0], n[-1], rtol=1e-14)


def test_action_latency_replays_shifted_actions():
    K = 5
    acts = np.stack([np.full((1, 4), HOVER * (0.95 + 0.02 * k)) for k in range(K)])
    xa, _ = _run(_level(), acts, dr=_dr(depth=3, delay=2), flags=oracle.GND | oracle.DRAG)
    applied = acts[[0, 0, 0, 1, 2]]
    xb, _ = _run(_level(), applied, flags=oracle.GND | oracle.DRAG)
    np.testing.assert_array_equal(xa, xb)


def test_steady_wind_drag():
    k, vw = 0.01, np.array([2.0, -1.0, 0.0])
    x, _ = _run(_level(), np.full((1, 1, 4), HOVER), dr=_dr(wind=oracle.WIND_CONSTANT, vwind=vw, kdrag=k))
    F = k * np.linalg.norm(vw) * vw
    np.testing.assert_allclose(x[0, 7:10], F / P.mass * P.dt_ctrl, rtol=1e-12, atol=1e-15)


def test_sinusoidal_wind_closed_form():
    A, w, K = 0.01, 2.0, 4
    x, _ = _run(_level(), np.full((K, 1, 4), HOVER), dr=_dr(wind=oracle.WIND_SINUSOIDAL, sin_a=A, sin_w=w))
    t = np.arange(K) * P.dt_ctrl
    F = A * np.stack([np.sin(w * t), np.cos(w * t), 0.3 * np.sin(2 * w * t)], axis=1)
    np.testing.assert_allclose(x[0, 7:10], F.sum(axis=0) / P.mass * P.dt_ctrl, rtol=1e-10, atol=1e-15)


def _dryden_series(sigma, V, h, steps, seed=5):
    row = oracle.neutral_dr(1)[0]
    row[oracle.DR_WIND] = oracle.WIND_DRYDEN
    row[oracle.DR_DRY_SIGMA], row[oracle.DR_DRY_V], row[oracle.DR_DRY_H] = sigma, V, h
    ws = np.zeros(oracle.WIND_STATE)
    ws[3] = -1.0
    xs = np.zeros((steps, 3))
    for i in range(steps):
        _, v = oracle.wind_step(P, row, ws, seed, 0)
        xs[i] = v
    return xs


def test_dryden_stationary_statistics():
    """x_t = alpha x_{t-1} + sigma sqrt(1 - alpha^2) xi: stationary variance sigma^2, lag-one
    correlation alpha, Gaussian innovations. Started at 0, so the first 5 time constants
    are dropped."""
    sigma, V, h = 0.5, 8.0, 2.0
    L = h / (0.177 + 8.23e-4 * h) ** 1.2
    alpha = np.exp(-P.dt_ctrl * V / L)
    xs = _dryden_series(sigma, V, h, 60000)[int(5 / (1 - alpha)):]
    n_eff = xs.shape[0] * (1 - alpha) / (1 + alpha)
    assert np.all(np.abs(xs.mean(axis=0)) < 4 * sigma / np.sqrt(n_eff))
    np.testing.assert_allclose(xs.var(axis=0), sigma ** 2, rtol=6 * np.sqrt(2 / n_eff))
    for r in range(3):
        rho = np.corrcoef(xs[:-1, r], xs[1:, r])[0, 1]
        assert rho == pytest.approx(alpha, abs=4 * np.sqrt((1 - alpha ** 2) / xs.shape[0]))  # AR(1) standard error
        xi = (xs[1:, r] - alpha * xs[:-1, r]) / (sigma * np.sqrt(1 - alpha ** 2))
        from scipy import stats
        assert stats.kstest(xi, "norm").pvalue > 1e-3


def _gust_row(p, A, T):
    row = oracle.neutral_dr(1)[0]
    row[oracle.DR_WIND] = oracle.WIND_GUST
    row[oracle.DR_GUST_P], row[oracle.DR_GUST_A], row[oracle.DR_GUST_T] = p, A, T
    return row


def test_gust_envelope():
    """p = 1, duration 4 control steps: a gust starts at once with phase 0, the force along a
    fixed unit direction is A sin(pi s) at s = 0, 1/4, ..., 1, then the next gust starts."""
    A = 0.2
    row = _gust_row(1.0, A, 4 * P.dt_ctrl)
    ws = np.zeros(oracle.WIND_STATE)
    ws[3] = -1.0
    F = np.array([oracle.wind_step(P, row, ws, 3, 7)[0] for _ in range(10)])
    mags = np.linalg.norm(F, axis=1)
    s = np.array([0, 0.25, 0.5, 0.75, 1.0, 0, 0.25, 0.5, 0.75, 1.0])
    np.testing.assert_allclose(mags, A * np.sin(np.pi * s), atol=1e-7)  # the phase advances in float32
    d1 = F[1:4] / mags[1:4, None]
    np.testing.assert_allclose(d1, np.repeat(d1[:1], 3, axis=0), atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(d1, axis=1), 1.0, atol=1e-12)
    assert not np.allclose(F[6] / mags[6], d1[0])  # a new direction for the next gust
    ws[3] = -1.0
    assert np.all([np.linalg.norm(oracle.wind_step(P, _gust_row(0.0, A, 1.0), ws, 3, 7)[0]) == 0 for _ in range(50)])


def test_gust_trigger_rate_and_direction():
    """Gusts shorter than a control step: every step starts idle, so the starts are
    Bernoulli(p); their directions are uniform on the sphere (mean 0, E[z^2] = 1/3)."""
    p, N = 0.25, 20000
    row = _gust_row(p, 1.0, 0.5 * P.dt_ctrl)
    ws = np.zeros(oracle.WIND_STATE)
    ws[3] = -1.0
    dirs, prev = [], ws[4:7].copy()
    for _ in range(N):
        oracle.wind_step(P, row, ws, 11, 2)
        assert ws[3] == -1.0  # over within its own step
        if not np.array_equal(ws[4:7], prev):  # a start draws a new direction
            dirs.append(ws[4:7].copy())
            prev = ws[4:7].copy()
    starts = len(dirs)
    assert abs(starts - p * N) < 4 * np.sqrt(N * p * (1 - p))
    D = np.array(dirs)
    np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-12)
    assert np.all(np.abs(D.mean(axis=0)) < 4 / np.sqrt(3 * len(D)))
    assert np.mean(D[:, 2] ** 2) == pytest.approx(1 / 3, abs=4 * np.sqrt(4 / 45 / len(D)))


def test_splitmix64_published_sequence():
    """SplitMix64 (Steele, Lea and Flood 2014) from state 0: the reference implementation's
    first outputs are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
    0xF88BB8A8724C81EC. A wrong constant, shift or increment in the oracle's round fails
    here (the input generator's copy is a second implementation, not a pin)."""
    gamma = 0x9E3779B97F4A7C15
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [oracle.splitmix64(k * gamma) for k in range(4)] == published
    # orc_uniform is five rounds over the counters, the top 24 bits scaled to [0, 1)
    h = oracle.splitmix64(0)
    for field in (21, 0, 0, 0):
        h = oracle.splitmix64(h ^ field)
    assert oracle.uniform(0, 21, 0, 0, 0) == (h >> 40) / 2.0 ** 24


def test_uniforms_match_the_input_generator():
    for seed, stream, step, index, comp in ((0, 21, 0, 0, 0), (7, 21, 3, 12, 4), (2 ** 40 + 3, 5, 99, 7, 6)):
        u = oracle.uniform(seed, stream, step, index, comp)
        v = wl.uniform(seed, stream, step, np.uint64(index), np.uint64(comp))
        assert u == float(v)


def _obs_run(P, x0, rpm, r, K=1):
    n = x0.shape[0]
    env_off = np.arange(n + 1, dtype=np.int32)
    return oracle.control_steps(P, env_off, np.zeros(n, np.int32), np.full(n, oracle.ACT_RPM, np.int32), x0,
                                np.zeros((n, 6)), np.zeros((n, 4)), np.repeat(rpm[None], K, axis=0), 5, obs=True, dr=r)


def test_observation_noise_statistics():
    """2000 identical drones with the table's sensor sigmas: the KIN observation minus the
    noiseless one, divided by the sigma, is standard normal and uncorrelated per channel;
    quaternion and RPM channels carry no noise."""
    n = 2000
    x0 = np.repeat(_level(z=1.0), n, axis=0)
    rpm = np.full((n, 4), HOVER)
    sig = {oracle.DR_NOISE_P: 0.01, oracle.DR_NOISE_V: 0.05, oracle.DR_NOISE_RPY: np.radians(1.0),
           oracle.DR_NOISE_W: 0.05}
    r0 = oracle.Randomization(n, n, 1, seed=3)
    r1 = oracle.Randomization(n, n, 1, seed=3)
    for col, v in sig.items():
        r1.env_dr[:, col] = v
    k0 = _obs_run(P, x0, rpm, r0)[3]
    k1 = _obs_run(P, x0, rpm, r1)[3]
    d = k1 - k0
    np.testing.assert_array_equal(d[:, 3:7], 0.0)
    np.testing.assert_array_equal(d[:, 16:20], 0.0)
    z = np.concatenate([d[:, 0:3] / 0.01, d[:, 7:10] / np.radians(1.0), d[:, 10:13] / 0.05, d[:, 13:16] / 0.05], axis=1)
    assert np.all(np.abs(z.mean(axis=0)) < 4 / np.sqrt(n))
    np.testing.assert_allclose(z.std(axis=0), 1.0, atol=4 / np.sqrt(2 * n))
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(12))) < 4 / np.sqrt(n)


def test_sensor_delay_reports_the_step_start():
    """With a one-step sensor delay (and no noise) the KIN observation after a control step is
    the one of the state and RPMs at the step's start; the neighbour observation is not
    delayed. Two steps: the second reports the state after the first."""
    x0 = np.stack([_level(z=1.0)[0], _level(z=1.3)[0]])
    x0[1, 0] = 0.2
    env_off = np.array([0, 2], np.int32)
    r = oracle.Randomization(1, 2, 1)
    r.env_dr[0, oracle.DR_OBS_DELAY] = 1.0
    rpm = np.array([[14000.0, 15000.0, 14500.0, 14800.0], [15500.0, 15000.0, 15200.0, 14900.0]])
    args = (env_off, np.zeros(1, np.int32), np.array([oracle.ACT_RPM], np.int32))
    a0 = np.full((2, 4), 123.0)
    x1, i1, a1, kin, idx, rel = oracle.control_steps(P, *args, x0, np.zeros((2, 6)), a0, rpm[None], 5, obs=True, dr=r)
    for j in range(2):
        np.testing.assert_array_equal(kin[j], oracle.kin(x0[j], a0[j]))
        i_ref, r_ref = oracle.knn(x1, j, 0)
        np.testing.assert_array_equal(idx[j], i_ref)
        np.testing.assert_allclose(rel[j], r_ref, rtol=1e-12)
    r2 = oracle.Randomization(1, 2, 1)
    r2.env_dr[0, oracle.DR_OBS_DELAY] = 1.0
    x2, _, a2, kin2, _, _ = oracle.control_steps(P, *args, x0, np.zeros((2, 6)), a0, np.repeat(rpm[None], 2, axis=0),
                                                 5, obs=True, dr=r2)
    for j in range(2):
        np.testing.assert_array_equal(kin2[j], oracle.kin(x1[j], a1[j]))


def test_observation_noise_changes_with_the_step():
    n = 50
    x0 = np.repeat(_level(z=1.0), n, axis=0)
    rpm = np.full((n, 4), HOVER)
    r = oracle.Randomization(n, n, 1, seed=8)
    r.env_dr[:, oracle.DR_NOISE_P] = 0.01
    k1 = _obs_run(P, x0, rpm, r)[3]
    k2 = _obs_run(P, x0, rpm, r)[3]  # same start, wind step counter advanced by one
    assert np.all(np.abs(k1[:, 0] - k2[:, 0]) > 0)
    r2 = oracle.Randomization(n, n, 1, seed=8)
    r2.env_dr[:, oracle.DR_NOISE_P] = 0.01
    np.testing.assert_array_equal(_obs_run(P, x0, rpm, r2)[3], k1)


# ---- episode reset: the "init" row and the sticky observation bias (Section 3.5) ----

INIT = (0.2, 0.1, 0.5)  # the table's init row: p0 m, RPY0 rad, v0 m/s
NOMINAL = (1.0, -2.0, 1.5, 0.7)


def _rot_zyx(roll, pitch, yaw):
    cr, sr, cp, sp, cy, sy = np.cos(roll), np.sin(roll), np.cos(pitch), np.sin(pitch), np.cos(yaw), np.sin(yaw)
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def test_reset_state_is_the_nominal_pose_plus_the_drawn_perturbation():
    """Each component is nominal + r (2u - 1) of its own counter-based uniform (stream 23):
    position and velocity directly, the attitude as the rotation Rz(yaw) Ry(pitch) Rx(roll)
    of the perturbed angles (built here as matrices; the oracle composes quaternions), at
    rest in rotation; the reset is a function of (seed, episode, drone) alone."""
    for drone in (0, 5, 12345):
        x = oracle.reset_state(NOMINAL, INIT, 9, 3, drone)
        u = np.array([2 * oracle.uniform(9, 23, 3, drone, k) - 1 for k in range(9)])
        np.testing.assert_allclose(x[0:3], np.array(NOMINAL[:3]) + INIT[0] * u[0:3], rtol=0, atol=1e-15)
        np.testing.assert_allclose(x[7:10], INIT[2] * u[6:9], rtol=0, atol=1e-15)
        assert np.all(x[10:13] == 0)
        assert abs(np.linalg.norm(x[3:7]) - 1) < 1e-15
        R = oracle.rotation(x[3:7])
        np.testing.assert_allclose(R, _rot_zyx(INIT[1] * u[3], INIT[1] * u[4], NOMINAL[3] + INIT[1] * u[5]),
                                   rtol=0, atol=1e-15)
        np.testing.assert_allclose(oracle.rpy(x[3:7]), [INIT[1] * u[3], INIT[1] * u[4], NOMINAL[3] + INIT[1] * u[5]],
                                   rtol=0, atol=1e-14)
        assert np.array_equal(x, oracle.reset_state(NOMINAL, INIT, 9, 3, drone))
        assert not np.array_equal(x, oracle.reset_state(NOMINAL, INIT, 9, 4, drone))
        assert not np.array_equal(x, oracle.reset_state(NOMINAL, INIT, 10, 3, drone))


def test_reset_state_uniform_moments():
    """Over 20000 drones each perturbation is uniform on [-r, r]: inside the range, mean 0 and
    variance r^2/3 within 4 standard errors, and the roll/pitch/yaw read back from the
    quaternion follow the same law (yaw about its nominal value)."""
    n = 20000
    X = np.array([oracle.reset_state(NOMINAL, INIT, 1, 0, d) for d in range(n)])
    rpy = np.array([oracle.rpy(q) for q in X[:, 3:7]]) - np.array([0.0, 0.0, NOMINAL[3]])
    for vals, r in ((X[:, 0:3] - np.array(NOMINAL[:3]), INIT[0]), (rpy, INIT[1]), (X[:, 7:10], INIT[2])):
        z = vals / r
        assert np.all(np.abs(z) <= 1.0 + 1e-12)
        assert np.all(np.abs(z.mean(axis=0)) < 4 * np.sqrt(1 / 3 / n))
        # var of U[-1, 1] is 1/3; the variance of z^2 is 1/5 - 1/9
        assert np.all(np.abs((z ** 2).mean(axis=0) - 1 / 3) < 4 * np.sqrt((1 / 5 - 1 / 9) / n))
    # the nine components are drawn independently
    C = np.corrcoef(np.concatenate([X[:, 0:3], rpy, X[:, 7:10]], 1).T)
    assert np.max(np.abs(C - np.eye(9))) < 4 / np.sqrt(n)


def test_obs_bias_gaussian_per_channel():
    """b_k = sigma[k // 3] xi_k with xi standard normal (Box-Muller, stream 24): per channel
    mean 0 and variance sigma^2 within 4 standard errors, a Kolmogorov-Smirnov test against
    the normal law, uncorrelated channels; a zero sigma gives zero channels."""
    from scipy import stats
    n = 20000
    sig = np.array([0.01, np.deg2rad(1.0), 0.05, 0.05])
    B = np.array([oracle.obs_bias(sig, 4, 2, d) for d in range(n)])
    Z = B / np.repeat(sig, 3)[None, :]
    assert np.all(np.abs(Z.mean(axis=0)) < 4 / np.sqrt(n))
    assert np.all(np.abs(Z.var(axis=0) - 1) < 4 * np.sqrt(2 / n))
    for k in range(12):
        assert stats.kstest(Z[:, k], "norm").pvalue > 1e-4
    C = np.corrcoef(Z.T)
    assert np.max(np.abs(C - np.eye(12))) < 4 / np.sqrt(n)
    b = oracle.obs_bias([0.0, 1.0, 0.0, 0.0], 4, 2, 7)
    assert np.all(b[0:3] == 0) and np.all(b[6:12] == 0) and np.all(b[3:6] != 0)
    assert np.array_equal(oracle.obs_bias(sig, 4, 2, 7), oracle.obs_bias(sig, 4, 2, 7))
    assert not np.array_equal(oracle.obs_bias(sig, 4, 2, 7), oracle.obs_bias(sig, 4, 3, 7))


def test_obs_bias_is_sticky_on_the_noisy_kin_channels():
    """With the sensor noise off, the KIN observation under a bias differs from the one
    without by exactly the bias, on position, roll/pitch/yaw, velocity and body rate, at
    every step of the episode (the same bias); quaternion and RPMs carry none; the state is
    untouched."""
    P = oracle.cf2x()
    n = 6
    x0 = np.array([oracle.reset_state(NOMINAL, INIT, 2, 0, d) for d in range(n)])
    rpm = np.full((n, 4), oracle.hover_rpm(P))
    bias = np.array([oracle.obs_bias([0.01, 0.02, 0.05, 0.05], 2, 0, d) for d in range(n)])
    env_off = np.arange(n + 1, dtype=np.int32)
    args = (P, env_off, np.zeros(n, np.int32), np.full(n, oracle.ACT_RPM, np.int32))
    outs = []
    for b in (None, bias):
        r = oracle.Randomization(n, n, 1, 3)
        r.obs_bias = b
        x, integ, a = x0, np.zeros((n, 6)), np.zeros((n, 4))
        ks = []
        for _ in range(2):
            x, integ, a, kin, _, _ = oracle.control_steps(*args, x, integ, a, rpm[None], 5, obs=True, dr=r)
            ks.append((x.copy(), kin))
        outs.append(ks)
    for (xa, ka), (xb, kb) in zip(*outs):
        assert np.array_equal(xa, xb)
        d = kb - ka
        np.testing.assert_allclose(d[:, 0:3], bias[:, 0:3], rtol=0, atol=1e-15)
        np.testing.assert_allclose(d[:, 7:10], bias[:, 3:6], rtol=0, atol=1e-15)
        np.testing.assert_allclose(d[:, 10:13], bias[:, 6:9], rtol=0, atol=1e-15)
        np.testing.assert_allclose(d[:, 13:16], bias[:, 9:12], rtol=0, atol=1e-15)
        assert np.all(d[:, 3:7] == 0) and np.all(d[:, 16:20] == 0)
