"""GPU parity of the model and integrator variants against the oracle: fourth-order
Runge-Kutta substeps (MDG_INTEGRATOR_RK4), the + rotor layout (CF2P) and the RACE model.

Same protocol as test_gpu_parity.py: the oracle, configured like the library, restarts
from the GPU's own float32 state; one substep is compared with the per-substep tolerances
(for RK4 with downwash, plus the oracle's measured response, since its stage states are
rounded to float32), one control step with the horizon bound
(helpers.assert_horizon_close), and the observations against the GPU's post-step state.

RK4 is compared drone by drone on well-conditioned batches: the dense and uneven recipes
keep their environment sizes, physics flags, action types and tiling, but every
environment's drones fly at distinct heights 0.3 m apart. In the recipes as drawn, pairs at
near-equal heights put the downwash (force ~ 1/dz^2, cut off at dz = 0) on a discontinuity:
the oracle itself, restarted from states moved by 1e-7 relative, spreads such drones over
hundreds of m/s within one control step. Those batches are compared under RK4 as ensembles
over long rollouts (test_gpu_statistics.py).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import (assert_horizon_close, assert_knn_valid, assert_state_close, oracle_arrays, oracle_step, spread_heights,
                     tolerance_response)

pytestmark = pytest.mark.gpu


def _pair(model, rk4):
    """(library constants, oracle parameters) of a model, with the chosen integrator."""
    c = getattr(mdg.Constants, model)()
    P = getattr(oracle, model)()
    if rk4:
        c.integrator = mdg.INTEGRATOR_RK4
        P.integrator = oracle.RK4
    return c, P


def _swarm(recipe):
    if recipe == "single":
        return wl.single(3, n_envs=100)
    if recipe == "full_aero":
        return wl.full_aero(4, n_envs=160)
    if recipe == "dense":
        return wl.dense(5, n_envs=4)
    if recipe == "dense_spread":
        return spread_heights(wl.dense(5, n_envs=4))
    if recipe == "uneven_spread":
        return spread_heights(wl.uneven(6, n_envs=150))
    return wl.uneven(6, n_envs=150)


def _actions(sw, P, recipe, act_default):
    if recipe.startswith("uneven"):
        return wl.mixed_actions(sw, 7, 0, oracle.hover_rpm(P)), mdg.ACT_MIXED, sw.act_type
    if act_default == mdg.ACT_PID:
        return wl.waypoints(8, sw.n), mdg.ACT_PID, np.full(sw.n_envs, mdg.ACT_PID)
    return wl.rpm_actions(9, sw.n, 0, oracle.hover_rpm(P)), mdg.ACT_RPM, np.full(sw.n_envs, mdg.ACT_RPM)


def _check_obs(xg, ap, dpe, kin, idx, rel):
    env_off = np.concatenate([[0], np.cumsum(dpe)])
    kin, idx, rel = kin.cpu().numpy().astype(np.float64), idx.cpu().numpy(), rel.cpu().numpy().astype(np.float64)
    for e in range(len(dpe)):
        b, N = int(env_off[e]), int(dpe[e])
        for j in range(N):
            k_ref = oracle.kin(xg[b + j], ap[b + j])
            np.testing.assert_allclose(kin[b + j], k_ref, rtol=1e-6, atol=1e-6, err_msg=f"kin {b + j}")
            r_ref, _ = assert_knn_valid(xg[b:b + N], j, b, idx[b + j], what=f"neighbours of drone {b + j}")
            np.testing.assert_allclose(rel[b + j], r_ref, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("recipe", ["single", "full_aero", "dense_spread", "uneven_spread"])
@pytest.mark.parametrize("block", [None, 512])
def test_rk4_substep_and_control_step_match_oracle(cuda, recipe, block):
    """RK4 in its kernel variants (block None: the default size, <= 256 threads; 512: the
    any-size variant): one substep, then one control step of 5 substeps within the horizon
    bound, observations included."""
    sw = _swarm(recipe)
    c, P = _pair("cf2x", rk4=True)
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    if block is not None:
        if block < max(sw.drones_per_env):
            pytest.skip("block smaller than an environment")
        h.set_block_size(block)
    if recipe.startswith("uneven"):
        h.set_action_types(sw.act_type)
    action, act, acts = _actions(sw, P, recipe, mdg.ACT_PID if recipe == "full_aero" else mdg.ACT_RPM)
    layout = (sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    a_dev = torch.as_tensor(action, device=cuda)
    # one substep. Unlike an Euler substep, whose forces see exactly the restarted state,
    # RK4's stage states are rounded to float32 on the GPU, and the downwash at
    # near-coincident heights (force ~ 1/dz^2) amplifies that rounding; the bound adds the
    # oracle's own response to an initial error of the per-substep tolerance, as the
    # control-step comparisons do (single drones have no such coupling: plain tolerances)
    x0, i0, a0 = oracle_arrays(state)
    h.step(state, a_dev, act, 1)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    xo, _, _ = oracle_step(P, layout, x0, i0, a0, action, acts, 1)
    if recipe == "single":
        assert_state_close(xg, xo, what=f"rk4 {recipe} substep")
    else:
        resp = tolerance_response(P, layout, x0, i0, a0, action, acts, 1)
        assert_horizon_close(xg, xo, resp, 1, what=f"rk4 {recipe} substep")
    # one control step with observations, from the GPU's state
    x0, i0, a0 = oracle_arrays(state)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, a_dev, act, 5, kin, idx, rel)
    torch.cuda.synchronize()
    xg, ig, ag = oracle_arrays(state)
    xo, io, _ = oracle_step(P, layout, x0, i0, a0, action, acts, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, action, acts, 5)
    assert_horizon_close(xg, xo, resp, 5, what=f"rk4 {recipe} control step")
    _check_obs(xg, ag, sw.drones_per_env, kin, idx, rel)
    assert h.status()[0] in (mdg.OK, mdg.ERR_NONFINITE)


def test_rk4_rollout_matches_oracle(cuda):
    """The persistent rollout with RK4 substeps against the oracle."""
    sw = spread_heights(wl.uneven(10, n_envs=120))
    c, P = _pair("cf2x", rk4=True)
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    h.set_action_types(sw.act_type)
    actions = wl.mixed_actions(sw, 11, 0, oracle.hover_rpm(P))[None]
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    h.rollout(state, torch.as_tensor(actions[:1], device=cuda), mdg.ACT_MIXED, 5, 1)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    layout = (sw.drones_per_env, sw.flags)
    xo, _, _ = oracle_step(P, layout, x0, i0, a0, actions[0], sw.act_type, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, actions[0], sw.act_type, 5)
    assert_horizon_close(xg, xo, resp, 5, what="rk4 rollout")


@pytest.mark.parametrize("model", ["cf2p", "race"])
@pytest.mark.parametrize("recipe", ["full_aero", "uneven"])
def test_model_control_step_matches_oracle(cuda, model, recipe):
    """CF2P (+ layout: motor torques and the PID's inverse mixing) and RACE (its constants
    and gains) through one control step, compile-time variants included."""
    sw = _swarm(recipe)
    c, P = _pair(model, rk4=False)
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    if recipe == "uneven":
        h.set_action_types(sw.act_type)
    action, act, acts = _actions(sw, P, recipe, mdg.ACT_PID)
    layout = (sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, torch.as_tensor(action, device=cuda), act, 5, kin, idx, rel)
    torch.cuda.synchronize()
    xg, ig, ag = oracle_arrays(state)
    xo, io, ao = oracle_step(P, layout, x0, i0, a0, action, acts, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, action, acts, 5)
    assert_horizon_close(xg, xo, resp, 5, what=f"{model} {recipe}")
    # the PID's RPMs (plane 5) in thrust space, as in the PID parity test
    np.testing.assert_allclose(P.kf * ag.astype(np.float64) ** 2, P.kf * ao ** 2, rtol=0,
                               atol=1e-5 * P.kf * oracle.max_rpm(P) ** 2)
    _check_obs(xg, ag, sw.drones_per_env, kin, idx, rel)


def test_surrogate_step_with_rk4_falls_back_to_rk4(cuda):
    """With RK4 constants, a surrogate step whose environments are all out of distribution
    (a box that excludes everything) is the plain RK4 control step: the PID's RPMs and the
    fallback's RK4 substeps against the oracle's RK4 control step within the horizon bound."""
    sw = spread_heights(wl.full_aero(12, n_envs=32))
    c, _ = _pair("cf2x", rk4=True)
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    m = mdg.MLP(128, wl.mlp_init(1))
    z = np.zeros(mdg.MLP_IN, np.float32)
    m.set_normalization(z, z + 1, np.zeros(mdg.MLP_OUT, np.float32), np.ones(mdg.MLP_OUT, np.float32), z - 1, z - 1)
    s_sur = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    x0, i0, a0 = oracle_arrays(s_sur)
    wp = wl.waypoints(1, sw.n)
    nfb = torch.zeros(1, dtype=torch.int32, device=cuda)
    m.step(h, s_sur, torch.as_tensor(wp, device=cuda), mdg.ACT_PID, 5, 4.0, nfb)
    torch.cuda.synchronize()
    assert int(nfb) == sw.n_envs
    xg, ig, _ = oracle_arrays(s_sur)
    _, P = _pair("cf2x", rk4=True)
    layout = (sw.drones_per_env, sw.flags)
    acts = np.full(sw.n_envs, mdg.ACT_PID)
    xo, io, _ = oracle_step(P, layout, x0, i0, a0, wp, acts, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, wp, acts, 5)
    assert_horizon_close(xg, xo, resp, 5, what="RK4 fallback")
    assert h.status()[0] == mdg.OK


def _with_gnd_rotor(model, rk4):
    c, P = _pair(model, rk4)
    c.gnd_heights = mdg.GND_ROTOR
    P.gnd_heights = oracle.GND_ROTOR
    return c, P


@pytest.mark.parametrize("model, recipe, rk4", [
    ("cf2x", "single", False), ("cf2p", "single", False), ("race", "single", False), ("cf2x", "single", True),
    ("cf2x", "full_aero", False), ("cf2x", "uneven", False), ("cf2p", "uneven_spread", True)])
def test_per_rotor_ground_heights_match_oracle(cuda, model, recipe, rk4):
    """Eq. ground at each rotor's height (MDG_GND_ROTOR) through one substep and one control
    step. The single-drone recipe flies tilted drones 5 cm to 1 m above the ground, where
    the rotors' heights differ from the centre's by a sizeable fraction; there the result
    must also differ from the printed (centre-of-mass) model, so that the switch is seen to
    act."""
    sw = _swarm(recipe)
    c, P = _with_gnd_rotor(model, rk4)
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    if recipe.startswith("uneven"):
        h.set_action_types(sw.act_type)
    action, act, acts = _actions(sw, P, recipe, mdg.ACT_PID if recipe == "full_aero" else mdg.ACT_RPM)
    layout = (sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    a_dev = torch.as_tensor(action, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    h.step(state, a_dev, act, 1)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    xo, _, _ = oracle_step(P, layout, x0, i0, a0, action, acts, 1)
    if recipe == "single":
        assert_state_close(xg, xo, what=f"{model} per-rotor substep")
        Pc = getattr(oracle, model)()
        Pc.integrator = P.integrator
        xc, _, _ = oracle_step(Pc, layout, x0, i0, a0, action, acts, 1)
        # one substep separates the two models by ~8e-5 m/s (CF2.x) to ~6e-3 m/s (RACE)
        assert np.max(np.abs(xg[:, 9] - xc[:, 9])) > 5 * 1e-5, "per-rotor heights had no effect"
    else:
        resp = tolerance_response(P, layout, x0, i0, a0, action, acts, 1)
        assert_horizon_close(xg, xo, resp, 1, what=f"{model} {recipe} per-rotor substep")
    x0, i0, a0 = oracle_arrays(state)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, a_dev, act, 5, kin, idx, rel)
    torch.cuda.synchronize()
    xg, _, ag = oracle_arrays(state)
    xo, _, _ = oracle_step(P, layout, x0, i0, a0, action, acts, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, action, acts, 5)
    assert_horizon_close(xg, xo, resp, 5, what=f"{model} {recipe} per-rotor control step")
    _check_obs(xg, ag, sw.drones_per_env, kin, idx, rel)


def test_per_rotor_ground_heights_rollout(cuda):
    """The persistent rollout's per-rotor variant: 10 control steps of the single-drone
    recipe (no downwash: linear accumulation of the per-substep tolerance)."""
    sw = wl.single(13, n_envs=100)
    c, P = _with_gnd_rotor("cf2x", False)
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    hover = oracle.hover_rpm(P)
    acts = np.stack([wl.rpm_actions(14, sw.n, k, hover) for k in range(10)])
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    h.rollout(state, torch.as_tensor(acts, device=cuda), mdg.ACT_RPM, 5, 10)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    env_off = np.arange(sw.n + 1, dtype=np.int32)
    xo, _, _ = oracle.control_steps(P, env_off, np.asarray(sw.flags, np.int32), np.full(sw.n, oracle.ACT_RPM, np.int32),
                                    x0, i0, a0, acts.astype(np.float64), 5)
    assert_state_close(xg, xo, scale=50.0, what="per-rotor rollout")
