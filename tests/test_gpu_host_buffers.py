"""mdg_step_obs_host: the step kernel reads the actions from, and writes the observations
to, pinned host memory directly. Same kernel as mdg_step_obs, so the results on identical
inputs are bit-identical to the device-buffer call; buffers the device cannot address are
rejected by argument checks before anything is launched."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VP = ctypes.c_void_p


def _obs_buffers(n, device):
    return (torch.zeros((n, mdg.KIN_DIM), dtype=torch.float32, device=device),
            torch.zeros((n, mdg.NBR_K), dtype=torch.int32, device=device),
            torch.zeros((n, mdg.NBR_K * mdg.NBR_FEAT), dtype=torch.float32, device=device))


@pytest.mark.parametrize("recipe", ["full_aero", "uneven"])
def test_host_buffers_match_device_buffers(cuda, recipe):
    sw = wl.full_aero(31, n_envs=1024) if recipe == "full_aero" else wl.uneven(32, n_envs=512)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    hover = mdg.Constants.cf2x().hover_rpm()
    if recipe == "uneven":
        h.set_action_types(sw.act_type)
        act_type = mdg.ACT_MIXED
    else:
        act_type = mdg.ACT_PID
    s_dev = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    s_host = s_dev.clone()
    kd, idd, rd = _obs_buffers(sw.n, cuda)
    kh, ih, rh = (t.pin_memory() for t in _obs_buffers(sw.n, "cpu"))
    for step in range(3):
        a = wl.mixed_actions(sw, 40, step, hover) if recipe == "uneven" else wl.waypoints(41, sw.n)
        a_dev = torch.as_tensor(a, device=cuda)
        a_host = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h.step_obs(s_dev, a_dev, act_type, 5, kd, idd, rd)
        h.step_obs_host(s_host, a_host, act_type, 5, kh, ih, rh)
        torch.cuda.synchronize()
        assert torch.equal(s_dev, s_host), f"state differs after step {step}"
        assert torch.equal(kd.cpu(), kh) and torch.equal(idd.cpu(), ih) and torch.equal(rd.cpu(), rh)
    assert h.status()[0] == mdg.OK


def test_host_call_rejects_unmapped_buffers(cuda):
    sw = wl.full_aero(33, n_envs=64)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    before = state.clone()
    pageable = np.zeros((sw.n, 4), np.float32)
    kh, ih, rh = (t.pin_memory() for t in _obs_buffers(sw.n, "cpu"))
    kd, _, _ = _obs_buffers(sw.n, cuda)
    L = mdg.lib()
    stream = VP(torch.cuda.current_stream().cuda_stream)
    # pageable host memory as the action
    rc = L.mdg_step_obs_host(h._h, VP(state.data_ptr()), pageable.ctypes.data_as(VP), mdg.ACT_PID, 5,
                             VP(kh.data_ptr()), VP(ih.data_ptr()), VP(rh.data_ptr()), stream)
    assert rc == mdg.ERR_ARG and b"action_host" in L.mdg_last_error()
    # device memory where host memory is required
    a_host = torch.zeros((sw.n, 4), dtype=torch.float32).pin_memory()
    rc = L.mdg_step_obs_host(h._h, VP(state.data_ptr()), VP(a_host.data_ptr()), mdg.ACT_PID, 5,
                             VP(kd.data_ptr()), VP(ih.data_ptr()), VP(rh.data_ptr()), stream)
    assert rc == mdg.ERR_ARG and b"kin_host" in L.mdg_last_error()
    with pytest.raises(ValueError):
        h.step_obs_host(state, torch.zeros((sw.n, 4)), mdg.ACT_PID, 5, kh, ih, rh)
    torch.cuda.synchronize()
    assert torch.equal(state, before)
