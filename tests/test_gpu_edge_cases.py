"""GPU edge cases: empty and ragged batches, the largest environment, degenerate geometry,
non-finite state reporting and argument errors, each checked against the oracle where a
result exists."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import (assert_horizon_close, assert_knn_valid, assert_state_close, oracle_arrays, oracle_step, spread_heights,
                     tolerance_response)

pytestmark = pytest.mark.gpu

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)


def _t(a, dev, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def _level(ps, dev, v=None, w=None):
    ps = np.asarray(ps, np.float32)
    n = ps.shape[0]
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    return mdg.pack_state(ps, q, np.zeros((n, 3)) if v is None else v, np.zeros((n, 3)) if w is None else w,
                          device=dev)


def test_empty_batch_is_a_noop(cuda):
    h = mdg.Handle(np.zeros(0, np.int32), np.zeros(0, np.uint32))
    assert h.n == 0
    state = torch.zeros((6, 0, 4), device=cuda)
    act = torch.zeros((0, 4), device=cuda)
    h.step(state, act, mdg.ACT_RPM, 5)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, act, mdg.ACT_PID, 5, kin, idx, rel)
    h.obs(state, kin, idx, rel)
    h.pid(state, act, torch.zeros((0, 4), device=cuda))
    assert h.status()[0] == mdg.OK


def test_zero_drone_environments_interleaved(cuda):
    dpe = np.array([0, 3, 0, 0, 2, 0, 5, 0], np.int32)
    flags = np.full(len(dpe), mdg.GND | mdg.DRAG | mdg.DW, np.uint32)
    n = int(dpe.sum())
    p, q, v, w = wl.random_states(41, n, pos_scale=0.4)
    h = mdg.Handle(dpe, flags)
    state = mdg.pack_state(p, q, v, w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    action = wl.rpm_actions(41, n, 0, HOVER)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, _t(action, cuda), mdg.ACT_RPM, 1, kin, idx, rel)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    xo = oracle_step(P, (dpe, flags), x0, i0, a0, action, np.zeros(len(dpe)), 1)[0]
    assert_state_close(xg, xo, what="zero-drone envs")
    idx = idx.cpu().numpy()
    # env of 3 drones at 0..2, env of 2 at 3..4, env of 5 at 5..9: neighbours stay inside
    assert set(idx[0][idx[0] >= 0]) <= {1, 2} and (idx[0] == -1).sum() == 2
    assert set(idx[3][idx[3] >= 0]) == {4} and (idx[3] == -1).sum() == 3
    assert set(idx[5]) <= {6, 7, 8, 9}


def test_largest_environment(cuda):
    N = mdg.MAX_ENV_DRONES
    side = 11
    k = np.arange(N)
    ps = np.stack([(k % side) * 0.3, ((k // side) % side) * 0.3, 0.5 + (k // (side * side)) * 0.25], 1)
    ps += wl.uniform_range(-0.03, 0.03, 51, 1, 0, k.astype(np.uint64)[:, None], np.arange(3, dtype=np.uint64)[None])
    dpe = np.array([N], np.int32)
    flags = np.array([mdg.GND | mdg.DRAG | mdg.DW], np.uint32)
    h = mdg.Handle(dpe, flags)
    assert h.block_size == 1024
    state = _level(ps, cuda)
    x0, i0, a0 = oracle_arrays(state)
    action = wl.rpm_actions(51, N, 0, HOVER)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, _t(action, cuda), mdg.ACT_RPM, 5, kin, idx, rel)
    torch.cuda.synchronize()
    xg, _, ag = oracle_arrays(state)
    xo = oracle_step(P, (dpe, flags), x0, i0, a0, action, [0], 5)[0]
    spread = tolerance_response(P, (dpe, flags), x0, i0, a0, action, [0], 5)
    assert_horizon_close(xg, xo, spread, 5, what="1024-drone env")
    idx = idx.cpu().numpy()
    for j in (0, 17, 500, 1023):
        assert_knn_valid(xg, j, 0, idx[j], what=f"neighbours of drone {j}")
    with pytest.raises(mdg.MdgError):
        mdg.Handle(np.array([N + 1], np.int32), np.zeros(1, np.uint32))


def test_degenerate_geometry(cuda):
    # env 0: two drones at the same point (dz = 0: no downwash, distance-0 tie);
    # env 1: coaxial pair 0.6875 m apart (beta = 0); env 2: an inverted drone near the ground;
    # env 3: one drone alone.
    dz0 = -P.dw_c3 / P.dw_c2
    ps = np.array([[0, 0, 1], [0, 0, 1], [0.2, 0, 0.5], [0.2, 0, 0.5 + dz0], [1, 1, 0.01], [3, 3, 2]], np.float32)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (6, 1))
    q[4] = [0, 1, 0, 0]  # rolled by pi
    dpe = np.array([2, 2, 1, 1], np.int32)
    flags = np.full(4, mdg.GND | mdg.DRAG | mdg.DW, np.uint32)
    h = mdg.Handle(dpe, flags)
    state = mdg.pack_state(ps, q, np.zeros((6, 3)), np.zeros((6, 3)), device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    action = np.full((6, 4), HOVER, np.float32)
    kin, idx, rel = h.new_obs(cuda)
    h.step_obs(state, _t(action, cuda), mdg.ACT_RPM, 1, kin, idx, rel)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    xo = oracle_step(P, (dpe, flags), x0, i0, a0, action, np.zeros(4), 1)[0]
    assert_state_close(xg, xo, what="degenerate geometry")
    assert np.all(np.isfinite(xg))
    idx = idx.cpu().numpy()
    np.testing.assert_array_equal(idx[0], [1, -1, -1, -1])
    np.testing.assert_array_equal(idx[1], [0, -1, -1, -1])
    np.testing.assert_array_equal(idx[5], [-1, -1, -1, -1])
    assert np.all(rel.cpu().numpy()[5] == 0)
    # the inverted drone gets no ground effect: it falls at g plus the downward thrust
    assert xg[4, 9] < -P.g * P.dt_sim * 1.5


def test_nonfinite_state_is_reported(cuda):
    sw = wl.full_aero(61, n_envs=64)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    p = sw.p.copy()
    p[77, 2] = np.nan
    state = mdg.pack_state(p, sw.q, sw.v, sw.w, device=cuda)
    h.step(state, _t(wl.waypoints(61, sw.n), cuda), mdg.ACT_PID, 5)
    rc, bits, first = h.status()
    assert rc == mdg.ERR_NONFINITE and bits & mdg.STATUS_NONFINITE
    # comparisons with NaN are false, so the NaN height stays with drone 77 (its env-mates
    # skip it in the downwash sum)
    assert first == 77
    # the status word is cleared by the read
    h.step(state[:, :, :], _t(wl.waypoints(61, sw.n), cuda), mdg.ACT_PID, 5)
    rc2, _, _ = h.status()
    assert rc2 == mdg.ERR_NONFINITE  # the state itself is still NaN
    clean = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    h.step(clean, _t(wl.waypoints(61, sw.n), cuda), mdg.ACT_PID, 5)
    assert h.status() == (mdg.OK, 0, -1)


def test_argument_errors(cuda):
    sw = wl.full_aero(71, n_envs=8)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    act = torch.zeros((sw.n, 4), device=cuda)
    L = mdg.lib()
    sp = state.data_ptr()
    assert L.mdg_step(h._h, sp + 4, act.data_ptr(), 0, 5, None) == mdg.ERR_ARG
    assert "aligned" in L.mdg_last_error().decode()
    assert L.mdg_step(h._h, sp, act.data_ptr(), 0, 0, None) == mdg.ERR_ARG
    assert L.mdg_step(h._h, sp, act.data_ptr(), 9, 5, None) == mdg.ERR_ARG
    assert L.mdg_step(h._h, sp, act.data_ptr(), mdg.ACT_MIXED, 5, None) == mdg.ERR_ARG
    assert "mdg_set_action_types" in L.mdg_last_error().decode()
    assert L.mdg_step(h._h, sp, None, 0, 5, None) == mdg.ERR_ARG
    with pytest.raises(mdg.MdgError):
        h.set_block_size(48)
    with pytest.raises(mdg.MdgError):
        h.set_action_types(np.full(sw.n_envs, 7, np.uint8))
    big = mdg.Handle(np.array([64], np.int32), np.zeros(1, np.uint32))
    with pytest.raises(mdg.MdgError):
        big.set_block_size(32)
    with pytest.raises(ValueError):
        h.step(state[:, :-1].contiguous(), act, mdg.ACT_RPM, 5)


def test_exp_map_across_rotation_rates(cuda):
    # The kernel evaluates the exponential map by series in theta^2 = (|w| dt / 2)^2 up to
    # theta^2 = 0.1 (|w| ~ 151.8 rad/s at 240 Hz) and by sincosf above: sweep across the switch.
    rates = np.array([0.0, 1e-6, 1e-3, 1.0, 50.0, 150.0, 151.5, 151.8, 152.0, 153.0, 300.0, 1000.0, 5000.0])
    n = len(rates) * 8
    dirs = wl.uniform_range(-1, 1, 81, 2, 0, np.arange(n, dtype=np.uint64)[:, None], np.arange(3, dtype=np.uint64)[None])
    dirs = dirs.astype(np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    w = (dirs * np.repeat(rates, 8)[:, None]).astype(np.float32)
    p, q, v, _ = wl.random_states(81, n)
    h = mdg.Handle(np.ones(n, np.int32), np.zeros(n, np.uint32))
    state = mdg.pack_state(p, q, v, w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    action = np.full((n, 4), HOVER, np.float32)
    h.step(state, _t(action, cuda), mdg.ACT_RPM, 1)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    xo = oracle_step(P, (np.ones(n, np.int32), np.zeros(n)), x0, i0, a0, action, np.zeros(n), 1)[0]
    assert_state_close(xg, xo, what="exp map")
    np.testing.assert_allclose(np.linalg.norm(xg[:, 3:7], axis=1), 1.0, atol=3e-7)


def test_sync_reports_a_busy_stream_then_recovers(cuda):
    """Failure detection on the host: mdg_sync returns MDG_ERR_TIMEOUT while a stream is
    still busy (here a bounded device sleep of ~0.3 s stands in for a stuck worker), and OK
    once the work is done; the context stays usable throughout."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(int(0.3 * 2.07e9))
    assert mdg.sync(s, timeout_ms=20) == mdg.ERR_TIMEOUT
    assert b"still busy" in mdg.lib().mdg_last_error()
    assert mdg.sync(s, timeout_ms=10000) == mdg.OK
    assert mdg.sync(s, timeout_ms=0) == mdg.OK


def test_neighbour_ties_and_nonfinite_in_four_drone_environments(cuda):
    """The compile-time 4-drone path (a uniform all-effects batch): drones on exact squares
    tie pairwise (ties to the lower index), a coincident pair ties at distance 0, and a drone
    with a NaN position is left out of its environment-mates' lists."""
    n_envs = 64
    dpe = np.full(n_envs, 4, np.int32)
    flags = np.full(n_envs, mdg.GND | mdg.DRAG | mdg.DW, np.uint32)
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    p = np.zeros((4 * n_envs, 3), np.float32)
    for e in range(n_envs):
        p[4 * e:4 * e + 4, :2] = sq * (0.25 + 0.01 * e) + np.float32(3.0 * e)
        p[4 * e:4 * e + 4, 2] = 1.0
    p[4 * 1 + 3] = p[4 * 1 + 0]          # env 1: drones 0 and 3 coincide
    p[4 * 2 + 1, 0] = np.nan             # env 2: drone 1 has a NaN position
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (4 * n_envs, 1))
    h = mdg.Handle(dpe, flags)
    state = mdg.pack_state(p, q, np.zeros_like(p), np.zeros_like(p), device=cuda)
    kin, idx, rel = h.new_obs(cuda)
    action = np.full((4 * n_envs, 4), HOVER, np.float32)
    h.step_obs(state, _t(action, cuda), mdg.ACT_RPM, 1, kin, idx, rel)
    torch.cuda.synchronize()
    xg, _, _ = oracle_arrays(state)
    idx = idx.cpu().numpy()
    # level hover from rest keeps x and y, and every drone of an environment at one height
    np.testing.assert_array_equal(xg[:, :2][np.isfinite(xg[:, 0])], p[:, :2][np.isfinite(p[:, 0])])
    square = np.array([[1, 3, 2, -1], [0, 2, 3, -1], [1, 3, 0, -1], [0, 2, 1, -1]])
    for e in [0] + list(range(3, n_envs)):
        np.testing.assert_array_equal(idx[4 * e:4 * e + 4], np.where(square >= 0, square + 4 * e, -1),
                                      err_msg=f"env {e}")
        for j in range(4):
            assert_knn_valid(xg[4 * e:4 * e + 4], j, 4 * e, idx[4 * e + j], what=f"env {e} drone {j}")
    # env 1: 0 and 3 at distance 0 from each other
    b = 4
    np.testing.assert_array_equal(idx[b + 0], [b + 3, b + 1, b + 2, -1])
    np.testing.assert_array_equal(idx[b + 3], [b + 0, b + 1, b + 2, -1])
    # env 2: drone 1 is not listed by the others; its own list holds nothing finite
    b = 8
    np.testing.assert_array_equal(idx[b + 0], [b + 3, b + 2, -1, -1])
    np.testing.assert_array_equal(idx[b + 2], [b + 3, b + 0, -1, -1])
    np.testing.assert_array_equal(idx[b + 3], [b + 0, b + 2, -1, -1])
    np.testing.assert_array_equal(idx[b + 1], [-1, -1, -1, -1])
    rc, bits, first = h.status()
    assert rc == mdg.ERR_NONFINITE and first == b + 1


def test_results_do_not_depend_on_the_tile_size(cuda):
    """A drone's arithmetic is its own: every block size of one kernel variant gives the
    same bits (tiles of 8 to 64 environments of the compile-time four-drone variant; 128 and
    256 environments of the runtime one), and the two variants agree within the stated
    tolerances."""
    sw = spread_heights(wl.full_aero(71, n_envs=2048))  # no near-coincident heights: the variants stay close
    wp = _t(wl.waypoints(71, sw.n), cuda)
    init = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    out = {}
    for block in (32, 64, 128, 256, 512, 1024):
        h = mdg.Handle(sw.drones_per_env, sw.flags)
        h.set_block_size(block)
        st = init.clone()
        kin, idx, rel = h.new_obs(cuda)
        for _ in range(3):
            h.step_obs(st, wp, mdg.ACT_PID, 5, kin, idx, rel)
        torch.cuda.synchronize()
        assert h.status()[0] == mdg.OK
        out[block] = (st, kin, idx, rel)
    for group in ((32, 64, 128, 256), (512, 1024)):
        ref = out[group[0]]
        for b in group[1:]:
            for x, y in zip(out[b], ref):
                assert torch.equal(x, y), f"block {b} differs from block {group[0]}"
    a, b = out[64], out[1024]
    assert torch.equal(a[2], b[2])                      # neighbour indices: bit-exact decisions
    # the variants sum the downwash in different orders: within the per-substep tolerances
    # over the 15 substeps of the three control steps
    assert_state_close(oracle_arrays(a[0])[0], oracle_arrays(b[0])[0], scale=15, what="variants")
