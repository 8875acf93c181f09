"""GPU parity of the action types beyond RPM and PID (Table "Action types"): normalized
RPM, ONE_D_RPM, VEL and ATTITUDE, uniform and mixed per environment, through one control
step, the persistent rollout, the allocation-free entry point and the surrogate's
preparation and fallback.

Same protocol as test_gpu_parity.py: the oracle, restarted from the GPU's float32 state
(integrals included, set away from zero), is compared over one control step with the
horizon bound; the RPMs the action produced (plane 5) in thrust space; the PID integrals
(planes 3-4) within 1e-5; the observations against the GPU's post-step state.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import (assert_horizon_close, assert_knn_valid, excess, oracle_arrays, oracle_horizon, oracle_step, spread_heights,
                     tolerance_response)

pytestmark = pytest.mark.gpu

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)
HOVER_T = P.mass * P.g
EXT = [mdg.ACT_RPM_NORM, mdg.ACT_ONE_D_RPM, mdg.ACT_VEL, mdg.ACT_ATTITUDE]


def _state(sw, device, seed):
    """The swarm's state with PID integrals drawn away from zero (position U[-0.3, 0.3],
    attitude U[-0.05, 0.05])."""
    ip = wl.uniform_range(-0.3, 0.3, seed, 12, 0, np.arange(sw.n, dtype=np.uint64)[:, None],
                          np.arange(3, dtype=np.uint64)[None, :])
    ia = wl.uniform_range(-0.05, 0.05, seed, 13, 0, np.arange(sw.n, dtype=np.uint64)[:, None],
                          np.arange(3, dtype=np.uint64)[None, :])
    return mdg.pack_state(sw.p, sw.q, sw.v, sw.w, ip=ip, ia=ia, device=device)


def _check_obs(xg, ap, dpe, kin, idx, rel):
    env_off = np.concatenate([[0], np.cumsum(dpe)])
    kin, idx, rel = kin.cpu().numpy().astype(np.float64), idx.cpu().numpy(), rel.cpu().numpy().astype(np.float64)
    for e in range(len(dpe)):
        b, N = int(env_off[e]), int(dpe[e])
        for j in range(N):
            np.testing.assert_allclose(kin[b + j], oracle.kin(xg[b + j], ap[b + j]), rtol=1e-6, atol=1e-6)
            r_ref, _ = assert_knn_valid(xg[b:b + N], j, b, idx[b + j], what=f"neighbours of drone {b + j}")
            np.testing.assert_allclose(rel[b + j], r_ref, rtol=1e-6, atol=1e-8)


def _compare_step(cuda, sw, types, act_type, seed, what):
    action = wl.typed_actions(sw.drones_per_env, types, seed, 0, HOVER, HOVER_T)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    if act_type == mdg.ACT_MIXED:
        h.set_action_types(types)
    state = _state(sw, cuda, seed)
    x0, i0, a0 = oracle_arrays(state)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, torch.as_tensor(action, device=cuda), act_type, 5, kin, idx, rel)
    torch.cuda.synchronize()
    xg, ig, ag = oracle_arrays(state)
    layout = (sw.drones_per_env, sw.flags)
    xo, io, ao = oracle_step(P, layout, x0, i0, a0, action, types, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, action, types, 5)
    assert_horizon_close(xg, xo, resp, 5, what=what)
    np.testing.assert_allclose(P.kf * ag ** 2, P.kf * ao ** 2, rtol=0, atol=1e-5 * P.kf * oracle.max_rpm(P) ** 2,
                               err_msg=f"{what}: rpm")
    assert excess(ig, io, 1e-5) <= 1.0, f"{what}: integrals"
    _check_obs(xg, ag, sw.drones_per_env, kin, idx, rel)
    return h


@pytest.mark.parametrize("act", EXT)
@pytest.mark.parametrize("recipe", ["full_aero", "single"])
def test_uniform_action_type(cuda, act, recipe):
    sw = wl.full_aero(21, n_envs=256) if recipe == "full_aero" else wl.single(22, n_envs=100)
    _compare_step(cuda, sw, np.full(sw.n_envs, act, np.uint8), act, 23, f"{recipe} action {act}")


def test_mixed_action_types(cuda):
    """Every type in one batch (environments of 1 to 32 drones, mixed physics)."""
    sw = wl.uneven(24, n_envs=200)
    types = wl.all_action_types(25, sw.n_envs)
    assert set(np.unique(types)) == set(wl.ALL_ACTION_TYPES)
    _compare_step(cuda, sw, types, mdg.ACT_MIXED, 26, "mixed action types")


def test_mixed_action_types_rollout(cuda):
    """Three control steps in one persistent launch, an action set per step."""
    sw = wl.full_aero(27, n_envs=240)
    types = wl.all_action_types(28, sw.n_envs)
    K = 3
    actions = np.stack([wl.typed_actions(sw.drones_per_env, types, 29, k, HOVER, HOVER_T) for k in range(K)])
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(types)
    state = _state(sw, cuda, 30)
    x0, i0, a0 = oracle_arrays(state)
    h.rollout(state, torch.as_tensor(actions, device=cuda), mdg.ACT_MIXED, 5, K)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    states, resp = oracle_horizon(P, sw.drones_per_env, sw.flags, types, x0, i0, a0, actions, 5)
    assert_horizon_close(xg, states[-1], resp[-1], 5 * K, what="mixed rollout")


def test_mixed_action_types_noalloc_equals_step_obs(cuda):
    sw = wl.uneven(31, n_envs=150)
    types = wl.all_action_types(32, sw.n_envs)
    action = torch.as_tensor(wl.typed_actions(sw.drones_per_env, types, 33, 0, HOVER, HOVER_T), device=cuda)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(types)
    sa = _state(sw, cuda, 34)
    sb = sa.clone()
    ka, ia_, ra = h.new_obs(cuda)
    h.step_obs(sa, action, mdg.ACT_MIXED, 5, ka, ia_, ra)
    kb, ib, rb = h.new_obs(cuda)
    status = torch.zeros(2, dtype=torch.int32, device=cuda)
    VP = ctypes.c_void_p
    dpe = np.ascontiguousarray(sw.drones_per_env, np.int32)
    flg = np.ascontiguousarray(sw.flags, np.uint32)
    at = np.ascontiguousarray(types, np.uint8)
    rc = mdg.lib().mdg_step_obs_noalloc(None, sw.n_envs, dpe.ctypes.data_as(VP), flg.ctypes.data_as(VP),
                                        at.ctypes.data_as(VP), VP(sb.data_ptr()), VP(action.data_ptr()),
                                        mdg.ACT_MIXED, 5, VP(kb.data_ptr()), VP(ib.data_ptr()), VP(rb.data_ptr()),
                                        VP(status.data_ptr()), VP(torch.cuda.current_stream().cuda_stream))
    assert rc == mdg.OK, mdg.lib().mdg_last_error()
    torch.cuda.synchronize()
    assert torch.equal(sa, sb) and torch.equal(ka, kb) and torch.equal(ia_, ib) and torch.equal(ra, rb)


def test_surrogate_fallback_with_every_action_type(cuda):
    """The surrogate step's preparation converts every action type; with every environment
    out of distribution the fallback's control step matches the oracle."""
    sw = wl.full_aero(35, n_envs=300)
    types = wl.all_action_types(36, sw.n_envs)
    action = wl.typed_actions(sw.drones_per_env, types, 37, 0, HOVER, HOVER_T)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(types)
    m = mdg.MLP((sw.n + 127) // 128 * 128, wl.mlp_init(38))
    z = np.zeros(mdg.MLP_IN, np.float32)
    m.set_normalization(z, z + 1, np.zeros(mdg.MLP_OUT, np.float32), np.ones(mdg.MLP_OUT, np.float32), z - 1e30,
                        z + 1e30)
    state = _state(sw, cuda, 39)
    x0, i0, a0 = oracle_arrays(state)
    nfb = torch.zeros(1, dtype=torch.int32, device=cuda)
    m.step(h, state, torch.as_tensor(action, device=cuda), mdg.ACT_MIXED, 5, 0.0, nfb)
    torch.cuda.synchronize()
    assert int(nfb) == sw.n_envs
    xg, ig, _ = oracle_arrays(state)
    layout = (sw.drones_per_env, sw.flags)
    xo, io, _ = oracle_step(P, layout, x0, i0, a0, action, types, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, action, types, 5)
    assert_horizon_close(xg, xo, resp, 5, what="surrogate fallback, every action type")
    assert excess(ig, io, 1e-5) <= 1.0


def test_action_type_arguments_are_checked(cuda):
    sw = wl.full_aero(40, n_envs=4)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    for bad in (mdg.ACT_MIXED, 7, 255):
        with pytest.raises(mdg.MdgError):
            h.set_action_types(np.full(sw.n_envs, bad, np.uint8))
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    a = torch.zeros((sw.n, 4), device=cuda)
    with pytest.raises(mdg.MdgError):
        h.step(state, a, 7, 5)


# ------------------------------------------------------------------ DSL controller
PD = oracle.controller_dsl(oracle.cf2x())


def _dsl_oracle(layout, x, integ, a_prev, actions, types, sp, n_sub=5):
    """The oracle's DSL control steps (actions [K, n, 4]) from a state and setpoints; returns
    (x, integ, a_prev, sp) and the response to a tolerance-size error in x (see
    tolerance_response), with the same setpoints."""
    dpe, flags = layout
    env_off = np.concatenate([[0], np.cumsum(dpe)]).astype(np.int32)
    args = (env_off, np.asarray(flags, np.int32), np.asarray(types, np.int32))
    sa = np.ascontiguousarray(sp, np.float64).copy()
    xa, ia, aa = oracle.control_steps(PD, *args, x, integ, a_prev, np.asarray(actions, np.float64), n_sub, setpoint=sa)
    rng = np.random.default_rng(0)
    sgn = rng.choice([-1.0, 1.0], size=x.shape)
    x2 = x.copy()
    for sl, tol in ((slice(0, 3), 1e-5), (slice(7, 10), 1e-5), (slice(10, 13), 1e-4)):
        x2[:, sl] = x[:, sl] + sgn[:, sl] * tol * np.maximum(np.abs(x[:, sl]), 1.0)
    q = x[:, 3:7] + sgn[:, 3:7] * 2e-6
    x2[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    sb = np.ascontiguousarray(sp, np.float64).copy()
    xb, _, _ = oracle.control_steps(PD, *args, x2, integ, a_prev, np.asarray(actions, np.float64), n_sub, setpoint=sb)
    return (xa, ia, aa, sa), np.abs(xa - xb)


def _dsl_handle(sw, cuda, types=None):
    h = mdg.Handle(sw.drones_per_env, sw.flags, mdg.Constants.cf2x().with_dsl())
    if types is not None:
        h.set_action_types(types)
    sp = h.new_setpoints(cuda)
    h.set_setpoints(sp)
    return h, sp


@pytest.mark.parametrize("recipe", ["full_aero", "mixed"])
def test_dsl_control_steps(cuda, recipe):
    """Three control steps one launch each, the oracle restarted from the GPU's state and
    setpoints every step (the first step initialises the NaN setpoints). Heights spread per
    environment (helpers.spread_heights): the controller is under test here, not the
    downwash's conditioning at near-equal heights."""
    if recipe == "full_aero":
        sw = spread_heights(wl.full_aero(41, n_envs=200))
        types = np.full(sw.n_envs, mdg.ACT_PID, np.uint8)
        act_type = mdg.ACT_PID
    else:
        sw = spread_heights(wl.uneven(42, n_envs=150))
        types = wl.all_action_types(43, sw.n_envs)
        act_type = mdg.ACT_MIXED
    h, sp = _dsl_handle(sw, cuda, types if act_type == mdg.ACT_MIXED else None)
    state = _state(sw, cuda, 44)
    layout = (sw.drones_per_env, sw.flags)
    pid_rows = np.repeat(types == mdg.ACT_PID, sw.drones_per_env)
    for k in range(3):
        action = wl.typed_actions(sw.drones_per_env, types, 45, k, HOVER, PD.mass * PD.g)
        x0, i0, a0 = oracle_arrays(state)
        sp0 = sp.cpu().numpy().astype(np.float64)
        h.step(state, torch.as_tensor(action, device=cuda), act_type, 5)
        torch.cuda.synchronize()
        xg, ig, ag = oracle_arrays(state)
        (xo, io, ao, so), resp = _dsl_oracle(layout, x0, i0, a0, action[None], types, sp0)
        assert_horizon_close(xg, xo, resp, 5, what=f"dsl {recipe} step {k}")
        np.testing.assert_allclose(PD.kf * ag ** 2, PD.kf * ao ** 2, rtol=0,
                                   atol=1e-5 * PD.kf * oracle.max_rpm(PD) ** 2, err_msg=f"rpm step {k}")
        assert excess(ig, io, 1e-5) <= 1.0
        sg = sp.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(sg[pid_rows])) and np.all(np.isnan(sg[~pid_rows, 0]))
        assert excess(sg[pid_rows], so[pid_rows], 1e-6) <= 1.0, f"setpoints step {k}"


def test_dsl_rollout_carries_setpoints(cuda):
    sw = spread_heights(wl.full_aero(46, n_envs=160))
    K = 4
    h, sp = _dsl_handle(sw, cuda)
    state = _state(sw, cuda, 47)
    wp = wl.waypoints(48, sw.n)
    x0, i0, a0 = oracle_arrays(state)
    h.rollout(state, torch.as_tensor(wp, device=cuda), mdg.ACT_PID, 5, K)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    types = np.full(sw.n_envs, mdg.ACT_PID)
    (xo, _, _, so), resp = _dsl_oracle((sw.drones_per_env, sw.flags), x0, i0, a0,
                                       np.repeat(wp[None], K, axis=0), types, oracle.new_setpoints(sw.n))
    assert_horizon_close(xg, xo, resp, 5 * K, what="dsl rollout")
    assert excess(sp.cpu().numpy(), so, 1e-5) <= 1.0


@pytest.mark.parametrize("dsl", [False, True])
def test_standalone_controller_with_feed_forward(cuda, dsl):
    sw = wl.full_aero(49, n_envs=64)
    c = mdg.Constants.cf2x().with_dsl() if dsl else mdg.Constants.cf2x()
    P = PD if dsl else oracle.cf2x()
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    sp = h.new_setpoints(cuda)
    if dsl:
        h.set_setpoints(sp)
    state = _state(sw, cuda, 50)
    wp = wl.waypoints(51, sw.n)
    ff = np.zeros((sw.n, 4), np.float32)
    ff[:, 0:3] = wl.uniform_range(-2.0, 2.0, 52, 14, 0, np.arange(sw.n, dtype=np.uint64)[:, None],
                                  np.arange(3, dtype=np.uint64)[None, :])
    x0, i0, _ = oracle_arrays(state)
    rpm = torch.empty((sw.n, 4), device=cuda)
    pe = torch.empty((sw.n, 3), device=cuda)
    ye = torch.empty((sw.n,), device=cuda)
    h.pid(state, torch.as_tensor(wp, device=cuda), rpm, pe, ye, target_acc=torch.as_tensor(ff, device=cuda))
    torch.cuda.synchronize()
    _, ig, _ = oracle_arrays(state)
    rpm, pe, ye = rpm.cpu().numpy(), pe.cpu().numpy(), ye.cpu().numpy()
    sg = sp.cpu().numpy()
    for j in range(sw.n):
        r, e, y, integ, s = oracle.pid_ff(P, x0[j], i0[j], wp[j], a_ff=ff[j, 0:3],
                                          sp=oracle.new_setpoints(1)[0] if dsl else None)
        np.testing.assert_allclose(P.kf * rpm[j].astype(np.float64) ** 2, P.kf * r ** 2, rtol=0,
                                   atol=1e-5 * P.kf * oracle.max_rpm(P) ** 2)
        np.testing.assert_allclose(pe[j], e, rtol=1e-5, atol=1e-6)
        assert abs(ye[j] - y) < 1e-5
        assert excess(ig[j], integ, 1e-5) <= 1.0
        if dsl:
            assert excess(sg[j], s, 1e-6) <= 1.0


def test_dsl_surrogate_fallback(cuda):
    sw = spread_heights(wl.full_aero(53, n_envs=120))
    h, sp = _dsl_handle(sw, cuda)
    m = mdg.MLP((sw.n + 127) // 128 * 128, wl.mlp_init(54))
    z = np.zeros(mdg.MLP_IN, np.float32)
    m.set_normalization(z, z + 1, np.zeros(mdg.MLP_OUT, np.float32), np.ones(mdg.MLP_OUT, np.float32), z - 1e30,
                        z + 1e30)
    state = _state(sw, cuda, 55)
    wp = wl.waypoints(56, sw.n)
    x0, i0, a0 = oracle_arrays(state)
    m.step(h, state, torch.as_tensor(wp, device=cuda), mdg.ACT_PID, 5, 0.0)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    (xo, _, _, so), resp = _dsl_oracle((sw.drones_per_env, sw.flags), x0, i0, a0, wp[None],
                                       np.full(sw.n_envs, mdg.ACT_PID), oracle.new_setpoints(sw.n))
    assert_horizon_close(xg, xo, resp, 5, what="dsl surrogate fallback")
    assert excess(sp.cpu().numpy(), so, 1e-6) <= 1.0


def test_dsl_needs_setpoints(cuda):
    sw = wl.full_aero(57, n_envs=8)
    h = mdg.Handle(sw.drones_per_env, sw.flags, mdg.Constants.cf2x().with_dsl())
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    with pytest.raises(mdg.MdgError):
        h.step(state, torch.as_tensor(wl.waypoints(58, sw.n), device=cuda), mdg.ACT_PID, 5)
