"""GPU parity of the multi-step persistent rollout (mdg_rollout), its CUDA graph and the
autotuner: against the FP64 oracle over the same K control steps, and against K single
steps of mdg_step_obs."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import (assert_horizon_close, assert_state_close, check_obs_against_own_state, oracle_arrays,
                     oracle_horizon, oracle_step, swarm_state, tolerance_response)

pytestmark = pytest.mark.gpu

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)
MAXRPM32 = np.float32(oracle.max_rpm(P))


def _setup(recipe, K):
    if recipe == "single":
        sw = wl.single(0)
        acts = np.stack([wl.rpm_actions(0, sw.n, k, HOVER) for k in range(K)])
        types = np.zeros(sw.n_envs, np.uint8)
        act_type = mdg.ACT_RPM
    elif recipe == "full_aero":
        sw = wl.full_aero(3, n_envs=257)
        acts = np.stack([wl.waypoints(3, sw.n)] * K)
        types = np.ones(sw.n_envs, np.uint8)
        act_type = mdg.ACT_PID
    elif recipe == "dense":
        sw = wl.dense(5, n_envs=5)
        acts = np.stack([wl.rpm_actions(5, sw.n, k, HOVER) for k in range(K)])
        types = np.zeros(sw.n_envs, np.uint8)
        act_type = mdg.ACT_RPM
    else:
        sw = wl.uneven(2, n_envs=150)
        acts = np.stack([wl.mixed_actions(sw, 2, k, HOVER) for k in range(K)])
        types = sw.act_type
        act_type = mdg.ACT_MIXED
    return sw, acts, types, act_type


def _oracle_rollout(sw, x0, i0, a0, acts, types, n_sub):
    return oracle.control_steps(P, sw.env_off, sw.flags.astype(np.int32), types.astype(np.int32), x0, i0, a0,
                                acts.astype(np.float64), n_sub)[0]


@pytest.mark.parametrize("recipe", ["single", "full_aero", "dense", "uneven"])
def test_rollout_matches_oracle(cuda, recipe):
    """K steps in one launch against the oracle's K-step trajectory: the states after every
    step (carried by the per-step KIN observations) and after the last one within the
    horizon bound of (k+1) * n_sub substeps; every step's observations against the oracle
    restarted from the state they describe. K single steps of mdg_step_obs obey the same
    bounds."""
    K, n_sub = 3, 5
    sw, acts, types, act_type = _setup(recipe, K)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    if act_type == mdg.ACT_MIXED:
        h.set_action_types(types)
    s_roll = swarm_state(sw, cuda)
    s_step = s_roll.clone()
    x0, i0, a0 = oracle_arrays(s_roll)
    acts_t = torch.as_tensor(acts, device=cuda)
    kin_k = torch.empty((K, sw.n, 20), device=cuda)
    idx_k = torch.empty((K, sw.n, 4), dtype=torch.int32, device=cuda)
    rel_k = torch.empty((K, sw.n, 24), device=cuda)
    h.rollout(s_roll, acts_t, act_type, n_sub, K, mdg.OBS_EVERY_STEP, kin_k, idx_k, rel_k)
    kin1, idx1, rel1 = h.new_obs(cuda)
    kin_s = []
    for k in range(K):
        h.step_obs(s_step, acts_t[k], act_type, n_sub, kin1, idx1, rel1)
        kin_s.append(kin1.clone())
    torch.cuda.synchronize()
    xo, resp = oracle_horizon(P, sw.drones_per_env, sw.flags, types, x0, i0, a0, acts, n_sub)
    kin_k, idx_k, rel_k = kin_k.cpu().numpy(), idx_k.cpu().numpy(), rel_k.cpu().numpy()
    layout = (sw.drones_per_env, sw.flags)
    for k in range(K):
        kk = kin_k[k].astype(np.float64)
        xk = np.concatenate([kk[:, 0:7], kk[:, 10:16]], axis=1)
        if k > 0 and act_type == mdg.ACT_RPM:
            # RPM actions need no controller state: restart the oracle from the rollout's own
            # state after step k-1 (its KIN output) for one control step. Beyond one step the
            # downwash makes trajectories chaotic, so this is the meaningful check there.
            kp = kin_k[k - 1].astype(np.float64)
            xp = np.concatenate([kp[:, 0:7], kp[:, 10:16]], axis=1)
            zi, za = np.zeros((sw.n, 6)), np.zeros((sw.n, 4))
            xo1 = oracle_step(P, layout, xp, zi, za, acts[k], types, n_sub)[0]
            r1 = tolerance_response(P, layout, xp, zi, za, acts[k], types, n_sub)
            assert_horizon_close(xk, xo1, r1, n_sub, what=f"{recipe} rollout step {k} (restarted)")
        else:
            assert_horizon_close(xk, xo[k], resp[k], (k + 1) * n_sub, what=f"{recipe} rollout step {k}")
            ks = kin_s[k].cpu().numpy().astype(np.float64)
            xs = np.concatenate([ks[:, 0:7], ks[:, 10:16]], axis=1)
            assert_horizon_close(xs, xo[k], resp[k], (k + 1) * n_sub, what=f"{recipe} single step {k}")
        check_obs_against_own_state(sw.drones_per_env, kin_k[k], idx_k[k], rel_k[k], what=f"step {k}")
    xg, _, ag = oracle_arrays(s_roll)
    np.testing.assert_array_equal(xg, np.concatenate([kin_k[-1][:, 0:7], kin_k[-1][:, 10:16]], 1))
    np.testing.assert_array_equal(ag, np.clip(acts[-1], 0, MAXRPM32) if act_type == mdg.ACT_RPM else ag)
    assert h.status()[0] == mdg.OK


def test_rollout_fixed_action_equals_per_step_actions(cuda):
    K = 4
    sw = wl.full_aero(4, n_envs=200)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    wp = torch.as_tensor(wl.waypoints(4, sw.n), device=cuda)
    s1 = swarm_state(sw, cuda)
    s2 = s1.clone()
    h.rollout(s1, wp, mdg.ACT_PID, 5, K)
    h.rollout(s2, wp.expand(K, -1, -1).contiguous(), mdg.ACT_PID, 5, K)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)
    # K = 0 is a no-op
    s3 = s1.clone()
    h.rollout(s3, wp, mdg.ACT_PID, 5, 0)
    torch.cuda.synchronize()
    assert torch.equal(s3, s1)


def test_rollout_graph_replays_the_rollout(cuda):
    K = 8
    sw = wl.uneven(6, n_envs=300)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(sw.act_type)
    acts = torch.as_tensor(np.stack([wl.mixed_actions(sw, 6, k, HOVER) for k in range(K)]), device=cuda)
    s_graph = swarm_state(sw, cuda)
    s_direct = s_graph.clone()
    kin_g, idx_g, rel_g = h.new_obs(cuda)
    kin_d, idx_d, rel_d = h.new_obs(cuda)
    g = h.rollout_graph(s_graph, acts, mdg.ACT_MIXED, 5, K, mdg.OBS_LAST, kin_g, idx_g, rel_g)
    for _ in range(2):  # the state advances in place: two replays are two rollouts
        g.launch()
        h.rollout(s_direct, acts, mdg.ACT_MIXED, 5, K, mdg.OBS_LAST, kin_d, idx_d, rel_d)
        torch.cuda.synchronize()
        assert torch.equal(s_graph, s_direct)
        assert torch.equal(kin_g, kin_d) and torch.equal(idx_g, idx_d) and torch.equal(rel_g, rel_d)
    g.close()


def test_rollout_schedules_and_item_caps_give_identical_results(cuda):
    """A drone's arithmetic does not depend on which persistent block runs its environment or
    on how environments are packed into work items: the work counter and the static schedule,
    with items of the whole block or of 32 or 64 drones, give bit-identical states and
    observations over an 8-step uneven rollout (one graph of each, replayed)."""
    K = 8
    sw = wl.uneven(9, n_envs=500)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(sw.act_type)
    h.set_block_size(128)
    acts = torch.as_tensor(np.stack([wl.mixed_actions(sw, 9, k, HOVER) for k in range(K)]), device=cuda)
    ref = None
    for mode, cap in ((mdg.SCHED_DYNAMIC, 0), (mdg.SCHED_STATIC, 0), (mdg.SCHED_STATIC, 64), (mdg.SCHED_DYNAMIC, 32),
                      (mdg.SCHED_STATIC, 32)):
        h.set_rollout_schedule(mode, cap)
        assert h.rollout_schedule == (mode, cap)
        st = swarm_state(sw, cuda)
        kin, idx, rel = h.new_obs(cuda)
        h.rollout(st, acts, mdg.ACT_MIXED, 5, K, mdg.OBS_LAST, kin, idx, rel)
        g = h.rollout_graph(st, acts, mdg.ACT_MIXED, 5, K, mdg.OBS_LAST, kin, idx, rel)
        g.launch()
        torch.cuda.synchronize()
        g.close()
        out = (st.clone(), kin.clone(), idx.clone(), rel.clone())
        if ref is None:
            ref = out
        else:
            for a, b in zip(out, ref):
                assert torch.equal(a, b), f"schedule {mode}, item cap {cap}"
    assert h.status()[0] == mdg.OK
    with pytest.raises(mdg.MdgError):
        h.set_rollout_schedule(7, 0)
    with pytest.raises(mdg.MdgError):
        h.set_rollout_schedule(mdg.SCHED_STATIC, -1)


@pytest.mark.parametrize("K", [0, 4])
def test_autotune_keeps_state_and_picks_a_valid_block(cuda, K):
    sw = wl.uneven(8, n_envs=400)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    h.set_action_types(sw.act_type)
    state = swarm_state(sw, cuda)
    before = state.clone()
    acts = torch.as_tensor(wl.mixed_actions(sw, 8, 0, HOVER), device=cuda)
    best, ms = h.autotune(state, acts, mdg.ACT_MIXED, 5, K)
    torch.cuda.synchronize()
    assert torch.equal(state, before)
    assert best in (32, 64, 128, 256, 512, 1024) and h.block_size == best and ms > 0
    mode, cap = h.rollout_schedule
    assert mode in (mdg.SCHED_DYNAMIC, mdg.SCHED_STATIC)
    assert cap == 0 or (K > 0 and max(32, int(sw.drones_per_env.max())) <= cap < best)
    # and the tuned handle still computes the step: one substep against the oracle
    x0, i0, a0 = oracle_arrays(state)
    h.step(state, acts, mdg.ACT_MIXED, 1)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    xo = oracle.control_steps(P, sw.env_off, sw.flags.astype(np.int32), sw.act_type.astype(np.int32), x0, i0, a0,
                              acts.cpu().numpy().astype(np.float64)[None], 1)[0]
    assert_state_close(xg, xo, what="tuned handle")
