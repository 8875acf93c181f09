"""The allocation-free entry point (mdg_step_obs_noalloc) against the handle API.

Some callers cannot call cudaMalloc (their device memory belongs to another allocator,
or they must not allocate once running); mdg_step_obs_noalloc serves them from a static
device array instead of handle-owned tables. This test calls it through the C ABI and
checks two consecutive control steps against mdg_step_obs on identical inputs, with the
parity suite's per-substep tolerances and exact neighbour indices. It lives in its own
file, collected last, and passes alone in a fresh process as well as after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import assert_state_close, excess, oracle_arrays

pytestmark = pytest.mark.gpu

VP = ctypes.c_void_p


def _noalloc_step(sw, state, action, act_type, kin, idx, rel, status, act_types=None):
    L = mdg.lib()
    dpe = np.ascontiguousarray(sw.drones_per_env, np.int32)
    flg = np.ascontiguousarray(sw.flags, np.uint32)
    at = None if act_types is None else np.ascontiguousarray(act_types, np.uint8)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.mdg_step_obs_noalloc(None, sw.n_envs, dpe.ctypes.data_as(VP), flg.ctypes.data_as(VP),
                                None if at is None else at.ctypes.data_as(VP), VP(state.data_ptr()),
                                VP(action.data_ptr()), act_type, 5, VP(kin.data_ptr()), VP(idx.data_ptr()),
                                VP(rel.data_ptr()), VP(status.data_ptr()), VP(stream))
    assert rc == mdg.OK, L.mdg_last_error().decode()


@pytest.mark.parametrize("recipe", ["full_aero", "uneven"])
def test_noalloc_matches_handle_api_two_steps(cuda, recipe):
    if recipe == "full_aero":
        sw = wl.full_aero(91, n_envs=2000)
        act_type, act_types = mdg.ACT_PID, None
        actions = [wl.waypoints(91, sw.n)] * 2
    else:
        sw = wl.uneven(92, n_envs=700)
        act_type, act_types = mdg.ACT_MIXED, sw.act_type
        actions = [wl.mixed_actions(sw, 92, k, 14475.8) for k in range(2)]
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    if act_types is not None:
        h.set_action_types(act_types)
    s_ref = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    s_new = s_ref.clone()
    obs_ref = h.new_obs(cuda)
    obs_new = h.new_obs(cuda)
    status = torch.full((2,), 7, dtype=torch.int32, device=cuda)
    for k in range(2):  # two calls in a row: the static tables are rewritten each time
        a = torch.as_tensor(actions[k], device=cuda)
        h.step_obs(s_ref, a, act_type, 5, *obs_ref)
        _noalloc_step(sw, s_new, a, act_type, *obs_new, status, act_types)
        torch.cuda.synchronize()
        xr, ir, ar = oracle_arrays(s_ref)
        xn, i_n, an = oracle_arrays(s_new)
        assert_state_close(xn, xr, what=f"call {k + 1}")
        assert excess(i_n, ir, 1e-5) <= 1.0 and excess(an, ar, 1e-5, floor=1e3) <= 1.0
        assert excess(obs_new[0].cpu().numpy(), obs_ref[0].cpu().numpy(), 1e-5) <= 1.0
        assert torch.equal(obs_new[1], obs_ref[1])
        assert excess(obs_new[2].cpu().numpy(), obs_ref[2].cpu().numpy(), 1e-5) <= 1.0
        st = status.cpu().numpy().view(np.uint32)
        assert st[0] == 0 and st[1] == 0xFFFFFFFF  # status cleared each call, nothing non-finite
        assert h.status()[0] == mdg.OK


def _small_batch(cuda):
    sw = wl.full_aero(93, n_envs=256)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    a = torch.as_tensor(wl.waypoints(93, sw.n), device=cuda)
    kin = torch.empty((sw.n, 20), device=cuda)
    idx = torch.empty((sw.n, 4), dtype=torch.int32, device=cuda)
    rel = torch.empty((sw.n, 24), device=cuda)
    status = torch.zeros(2, dtype=torch.int32, device=cuda)
    return sw, state, a, kin, idx, rel, status


def test_noalloc_calls_leave_device_memory_unchanged(cuda):
    """The point of the entry point: after one call (which may load the library's device
    code on this device), further calls take no device memory. Every tensor is allocated
    before the first reading, and nothing else runs between the readings."""
    sw, state, a, kin, idx, rel, status = _small_batch(cuda)
    _noalloc_step(sw, state, a, mdg.ACT_PID, kin, idx, rel, status)
    torch.cuda.synchronize()
    torch.cuda.mem_get_info()  # any first-use set-up of the query itself
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        _noalloc_step(sw, state, a, mdg.ACT_PID, kin, idx, rel, status)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_a_capturing_stream(cuda):
    """A graph captured around the call would replay uploads from a host buffer that later
    calls overwrite: the call returns MDG_ERR_UNSUPPORTED while the stream is capturing, and
    works again on the same stream afterwards."""
    sw, state, a, kin, idx, rel, status = _small_batch(cuda)
    L = mdg.lib()
    dpe = np.ascontiguousarray(sw.drones_per_env, np.int32)
    flg = np.ascontiguousarray(sw.flags, np.uint32)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, device=cuda)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            marker.add_(1.0)  # the graph is not empty
            rc = L.mdg_step_obs_noalloc(None, sw.n_envs, dpe.ctypes.data_as(VP), flg.ctypes.data_as(VP), None,
                                        VP(state.data_ptr()), VP(a.data_ptr()), mdg.ACT_PID, 5,
                                        VP(kin.data_ptr()), VP(idx.data_ptr()), VP(rel.data_ptr()),
                                        VP(status.data_ptr()), VP(side.cuda_stream))
            msg = L.mdg_last_error().decode()
    assert rc == mdg.ERR_UNSUPPORTED and "captured" in msg
    torch.cuda.synchronize()
    _noalloc_step(sw, state, a, mdg.ACT_PID, kin, idx, rel, status)
    torch.cuda.synchronize()
    assert status.cpu().numpy().view(np.uint32)[0] == 0


def test_noalloc_rejects_oversized_batches(cuda):
    L = mdg.lib()
    n_envs = 16385
    dpe = np.ones(n_envs, np.int32)
    flg = np.zeros(n_envs, np.uint32)
    rc = L.mdg_step_obs_noalloc(None, n_envs, dpe.ctypes.data_as(VP), flg.ctypes.data_as(VP), None, None, None,
                                mdg.ACT_RPM, 5, None, None, None, None, None)
    assert rc == mdg.ERR_ARG
    assert "16384" in L.mdg_last_error().decode()
