"""GPU parity of domain randomization, motor lag, action latency and wind (Section 3.5).

Rows drawn from the paper's recommended ranges (workloads.dr_table, every wind model on).
Each control step, the oracle restarts from the GPU's state and randomization state
(rotor speeds, action history, wind state) and is compared over the step with the horizon
bound; the RPMs, integrals, rotor speeds and wind state against the oracle's, the action
history and the step counters exactly, the gust phases by check_gust_phases, the KIN
observation with its sensor noise and delay against the oracle's (the wind draws come from the
same counter-based SplitMix64 stream on both sides). Heights are spread per environment
(helpers.spread_heights): the randomization is under test, not the downwash's conditioning.

The gust phase advances by dt_ctrl/T per control step, in FP64 in the oracle and in float32
on the GPU, and a gust ends at the first step whose advanced phase exceeds 1. Where the
advanced phase lies within float32 rounding of 1 the two may end the gust one step apart;
both are correct. The force of that step is the same on both sides (it uses the phase before
the advance); only the next step's trigger may differ, and the tests restart the oracle from
the GPU's wind state each step.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import assert_horizon_close, excess, oracle_arrays, spread_heights

pytestmark = pytest.mark.gpu

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)
SEED = 77
DEPTH = 3


# float32 rounding of s + dt/T for s in [0, 1]: the sum's rounding (2^-24), the quotient's
# relative rounding and that of the float32 inputs (a few units of 2^-24 of dt/T <= 1): far
# below 1e-6.
PHASE_ATOL = 1e-6


def check_gust_phases(wg, wo, what):
    """Gust phases of the GPU (wg) and the oracle (wo) after the same step: idle (-1) on both
    sides or active on both within PHASE_ATOL, except a gust that one side ended and the other
    did not, which is valid only if the phase still running is within PHASE_ATOL of 1 (the
    end decision then rests on float32 rounding). Returns the environments where that
    happened."""
    ig, io = wg < 0, wo < 0
    assert np.all(wg[ig] == -1.0) and np.all(wo[io] == -1.0), f"{what}: idle phases"
    both = ~ig & ~io
    np.testing.assert_allclose(wg[both], wo[both], rtol=0, atol=PHASE_ATOL, err_msg=f"{what}: gust phases")
    split = np.flatnonzero(ig != io)
    running = np.where(ig[split], wo[split], wg[split])
    assert np.all(running >= 1.0 - PHASE_ATOL), f"{what}: gust ended on one side only at phases {running}"
    return split


def _oracle_state(table, motor, hist, wind, bias=None):
    r = oracle.Randomization(table.shape[0], motor.shape[0], hist.shape[0], SEED)
    r.env_dr[:] = table.astype(np.float64)
    r.motor[:] = motor.cpu().numpy().astype(np.float64)
    r.hist[:] = hist.cpu().numpy().astype(np.float64)
    r.wind[:] = wind.cpu().numpy().astype(np.float64)
    if bias is not None:
        r.obs_bias = np.ascontiguousarray(bias.cpu().numpy().astype(np.float64))
    return r


def _oracle_steps(sw, types, x, integ, a_prev, actions, r, perturb=False, obs=False):
    env_off = np.concatenate([[0], np.cumsum(sw.drones_per_env)]).astype(np.int32)
    if perturb:  # the horizon bound's response: an initial error of the per-substep tolerance
        rng = np.random.default_rng(0)
        sgn = rng.choice([-1.0, 1.0], size=x.shape)
        x = x.copy()
        for sl, tol in ((slice(0, 3), 1e-5), (slice(7, 10), 1e-5), (slice(10, 13), 1e-4)):
            x[:, sl] += sgn[:, sl] * tol * np.maximum(np.abs(x[:, sl]), 1.0)
        q = x[:, 3:7] + sgn[:, 3:7] * 2e-6
        x[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    return oracle.control_steps(P, env_off, sw.flags.astype(np.int32), np.asarray(types, np.int32), x, integ,
                                a_prev, np.asarray(actions, np.float64), 5, dr=r, obs=obs)


def _copy(r):
    c = oracle.Randomization(r.env_dr.shape[0], r.motor.shape[0], r.hist.shape[0], r.seed)
    for k in ("env_dr", "motor", "hist", "wind"):
        getattr(c, k)[:] = getattr(r, k)
    c.obs_bias = r.obs_bias
    return c


INIT = (0.2, 0.1, 0.5)  # the init row of the randomization table
BIAS_SIGMA = (0.01, float(np.deg2rad(1.0)), 0.05, 0.05)


def _bias(h, sw, cuda, episode=0):
    """A sticky observation bias drawn by mdg_reset (into a scratch state)."""
    scratch = torch.zeros((mdg.STATE_PLANES, sw.n, 4), device=cuda)
    nominal = torch.zeros((sw.n, 4), device=cuda)
    bias = torch.empty((sw.n, 12), device=cuda)
    h.reset(scratch, nominal, None, BIAS_SIGMA, bias, seed=SEED, episode=episode)
    return bias


def _setup(cuda, recipe):
    if recipe == "full_aero":
        sw = spread_heights(wl.full_aero(91, n_envs=160))
        types = np.full(sw.n_envs, mdg.ACT_PID, np.uint8)
    elif recipe == "mixed":
        sw = spread_heights(wl.uneven(92, n_envs=120))
        types = wl.all_action_types(93, sw.n_envs)
    else:
        sw = wl.single(94, n_envs=128)
        types = np.full(sw.n_envs, mdg.ACT_RPM, np.uint8)
    table = wl.dr_table(95, sw.n_envs, depth=DEPTH)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(types)
    motor, hist, wind = h.new_randomization_state(DEPTH, cuda)
    h.set_randomization(torch.as_tensor(table, device=cuda), motor, hist, wind, seed=SEED)
    bias = _bias(h, sw, cuda)
    h.set_obs_bias(bias)
    return sw, types, table, h, motor, hist, wind, bias


@pytest.mark.parametrize("recipe", ["full_aero", "mixed", "single"])
def test_randomized_control_steps(cuda, recipe):
    sw, types, table, h, motor, hist, wind, bias = _setup(cuda, recipe)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    kin, idx, rel = h.new_obs(cuda)
    for k in range(4):
        action = wl.typed_actions(sw.drones_per_env, types, 96, k, HOVER, P.mass * P.g)
        x0, i0, a0 = oracle_arrays(state)
        r = _oracle_state(table, motor, hist, wind, bias)
        r2 = _copy(r)
        h.step_obs(state, torch.as_tensor(action, device=cuda), mdg.ACT_MIXED, 5, kin, idx, rel)
        torch.cuda.synchronize()
        xg, ig, ag = oracle_arrays(state)
        xo, io, ao, ko, _, _ = _oracle_steps(sw, types, x0, i0, a0, action[None], r, obs=True)
        xp, _, _ = _oracle_steps(sw, types, x0, i0, a0, action[None], r2, perturb=True)
        what = f"{recipe} step {k}"
        assert_horizon_close(xg, xo, np.abs(xo - xp), 5, what=what)
        np.testing.assert_allclose(P.kf * ag ** 2, P.kf * ao ** 2, rtol=0, atol=1e-5 * P.kf * oracle.max_rpm(P) ** 2,
                                   err_msg=f"{what}: rpm")
        assert excess(ig, io, 1e-5) <= 1.0, f"{what}: integrals"
        assert excess(motor.cpu().numpy(), r.motor, 1e-5) <= 1.0, f"{what}: rotor speeds"
        np.testing.assert_array_equal(hist.cpu().numpy().astype(np.float64), r.hist, err_msg=f"{what}: history")
        wg = wind.cpu().numpy().astype(np.float64)
        check_gust_phases(wg[:, 3], r.wind[:, 3], what)
        np.testing.assert_array_equal(wg[:, 7], r.wind[:, 7], err_msg=f"{what}: wind steps")
        np.testing.assert_allclose(wg[:, 0:3], r.wind[:, 0:3], rtol=1e-4, atol=1e-5, err_msg=f"{what}: Dryden")
        np.testing.assert_allclose(wg[:, 4:7], r.wind[:, 4:7], rtol=0, atol=1e-6, err_msg=f"{what}: gust directions")
        # the KIN observation with sensor noise and delay (the oracle from the same start: a
        # delayed drone reports the step's start exactly; the others the end of the step,
        # within the step's tolerance) and the neighbour indices of the end-of-step state
        kg = kin.cpu().numpy().astype(np.float64)
        delayed = np.repeat(table[:, oracle.DR_OBS_DELAY] == 1, sw.drones_per_env)
        assert delayed.any() and (~delayed).any()
        np.testing.assert_allclose(kg[delayed], ko[delayed], rtol=1e-5, atol=1e-6, err_msg=f"{what}: delayed KIN")
        ok = ~delayed
        assert excess(kg[ok][:, 0:3], ko[ok][:, 0:3], 5 * 1e-5) <= 1.0, f"{what}: KIN position"
        assert np.max(np.abs(kg[:, 16:20] - ko[:, 16:20])) <= 1e-2, f"{what}: KIN RPMs"
        noise = kg[ok][:, 0:3] - xg[ok][:, 0:3] - bias.cpu().numpy()[ok][:, 0:3]  # the position noise the GPU added
        assert np.all(np.abs(noise) < 0.08) and np.std(noise) > 0.005, f"{what}: position noise"
    assert (wind[:, 3] >= 0).any(), "no gust was active during the test"
    assert h.status()[0] == mdg.OK


def test_randomized_rollout(cuda):
    sw, types, table, h, motor, hist, wind, bias = _setup(cuda, "full_aero")
    K = 4
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    actions = np.stack([wl.typed_actions(sw.drones_per_env, types, 97, k, HOVER, P.mass * P.g) for k in range(K)])
    x0, i0, a0 = oracle_arrays(state)
    r = _oracle_state(table, motor, hist, wind, bias)
    r2 = _copy(r)
    h.rollout(state, torch.as_tensor(actions, device=cuda), mdg.ACT_MIXED, 5, K)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    # the oracle one step at a time (the same as K steps in one call), recording the gusts
    # whose end fell within float32 rounding of a phase of 1: from there on the two sides may
    # follow different, equally valid gust sequences, so those environments leave the state
    # comparison (the seeds here give none; the assertion below says so)
    T = table[:, oracle.DR_GUST_T].astype(np.float64)
    xo, io, ao = x0, i0, a0
    ambiguous = np.zeros(sw.n_envs, bool)
    for k in range(K):
        s_next = r.wind[:, 3] + P.dt_ctrl / T
        ambiguous |= (r.wind[:, 3] >= 0) & (np.abs(s_next - 1.0) <= PHASE_ATOL)
        xo, io, ao = _oracle_steps(sw, types, xo, io, ao, actions[k:k + 1], r)
    xp, _, _ = _oracle_steps(sw, types, x0, i0, a0, actions, r2, perturb=True)
    assert ambiguous.sum() <= 1
    keep = ~np.repeat(ambiguous, sw.drones_per_env)
    assert_horizon_close(xg[keep], xo[keep], np.abs(xo - xp)[keep], 5 * K, what="randomized rollout")
    wg = wind.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(wg[:, 7], K)
    check_gust_phases(wg[~ambiguous, 3], r.wind[~ambiguous, 3], "randomized rollout")
    np.testing.assert_array_equal(hist.cpu().numpy().astype(np.float64), r.hist)


def test_randomization_arguments(cuda):
    sw = wl.full_aero(98, n_envs=8)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    motor, hist, wind = h.new_randomization_state(2, cuda)
    good = wl.dr_table(99, sw.n_envs, depth=2)
    for col, val in ((mdg.DR_MASS, 0.0), (mdg.DR_DELAY, 2.0), (mdg.DR_DELAY, 0.5), (mdg.DR_WIND, 16.0),
                     (mdg.DR_GUST_P, 1.5), (mdg.DR_GUST_T, 0.0), (mdg.DR_TAU, -0.01)):
        bad = good.copy()
        bad[3, col] = val
        with pytest.raises(mdg.MdgError):
            h.set_randomization(torch.as_tensor(bad, device=cuda), motor, hist, wind)
    h.set_randomization(torch.as_tensor(good, device=cuda), motor, hist, wind)
    h.set_randomization(None)
    c = mdg.Constants.cf2x()
    c.integrator = mdg.INTEGRATOR_RK4
    h4 = mdg.Handle(sw.drones_per_env, sw.flags, c)
    with pytest.raises(mdg.MdgError) as e:
        h4.set_randomization(torch.as_tensor(good, device=cuda), motor, hist, wind)
    assert e.value.code == mdg.ERR_UNSUPPORTED


def test_reset_matches_oracle(cuda):
    """mdg_reset against orc_reset_state / orc_obs_bias drone by drone: the drawn initial
    position, attitude and velocity (the init row of the randomization table) and the sticky
    bias, float32 against FP64 rounding; body rates, integrals and last RPMs zero; another
    episode draws another state, the same one the same state."""
    sw = wl.full_aero(98, n_envs=512)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    yaw = wl.uniform_range(-3.0, 3.0, 98, 40, 0, np.arange(sw.n, dtype=np.uint64), 0)
    nominal = np.concatenate([sw.p, yaw[:, None]], 1).astype(np.float32)
    state = torch.full((mdg.STATE_PLANES, sw.n, 4), float("nan"), device=cuda)
    bias = torch.empty((sw.n, 12), device=cuda)
    h.reset(state, torch.as_tensor(nominal, device=cuda), INIT, BIAS_SIGMA, bias, seed=SEED, episode=7)
    torch.cuda.synchronize()
    x, integ, a_prev = oracle_arrays(state)
    b = bias.cpu().numpy().astype(np.float64)
    xo = np.array([oracle.reset_state(nominal[g].astype(np.float64), INIT, SEED, 7, g) for g in range(sw.n)])
    bo = np.array([oracle.obs_bias(BIAS_SIGMA, SEED, 7, g) for g in range(sw.n)])
    np.testing.assert_allclose(x[:, 0:3], xo[:, 0:3], rtol=0, atol=1e-6)
    np.testing.assert_allclose(x[:, 3:7], xo[:, 3:7], rtol=0, atol=2e-6)
    np.testing.assert_allclose(x[:, 7:10], xo[:, 7:10], rtol=0, atol=1e-6)
    assert np.all(x[:, 10:13] == 0) and np.all(integ == 0) and np.all(a_prev == 0)
    np.testing.assert_allclose(b, bo, rtol=1e-5, atol=1e-7)
    again = torch.empty_like(state)
    h.reset(again, torch.as_tensor(nominal, device=cuda), INIT, None, None, seed=SEED, episode=7)
    other = torch.empty_like(state)
    h.reset(other, torch.as_tensor(nominal, device=cuda), INIT, None, None, seed=SEED, episode=8)
    torch.cuda.synchronize()
    assert torch.equal(again, state) and not torch.equal(other, state)
    with pytest.raises(mdg.MdgError):
        h.reset(state, torch.as_tensor(nominal, device=cuda), (0.2, -0.1, 0.5))
    with pytest.raises(mdg.MdgError):
        h.reset(state, torch.as_tensor(nominal, device=cuda), INIT, None, bias)


def test_obs_bias_needs_randomization(cuda):
    sw = wl.full_aero(99, n_envs=8)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    with pytest.raises(mdg.MdgError):
        h.set_obs_bias(torch.zeros((sw.n, 12), device=cuda))
