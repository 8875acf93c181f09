"""Index checks of the debug build.

compute-sanitizer is not available here, so the library has a debug build
(build_library(debug=True), -DMDG_DEBUG) whose kernels check every tile, environment and
list index they decode against its table (tile inside the batch and the block, whole
environments, the thread inside its environment, fallback entries inside the batch) and
record MDG_STATUS_BOUNDS instead of touching memory outside it. This test builds it and,
in a separate process that loads it, runs every kernel family on the workloads of the
parity suite (uniform and table tiles, compile-time and runtime environment sizes, the
persistent rollout, observations, PID, surrogate features, preparation, application and
the fallback pass, the allocation-free entry point, the RK4 and per-rotor ground-height
variants, every action type, randomization, the camera); no check may fail.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_debug_build_finds_no_index_outside_its_table(cuda):
    from paper_2606_08039_gb300 import build
    build.build_library(debug=True)
    env = dict(os.environ, MDG_DEBUG_LIBRARY="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--run"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all checks passed" in r.stdout


def _run():
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import workloads as wl
    assert mdg.LIB_PATH.endswith("libmdg_debug.so"), mdg.LIB_PATH
    dev = torch.device("cuda", 0)
    hover = mdg.Constants.cf2x().hover_rpm()
    seen = []

    def check(h, what):
        rc, bits, _ = h.status()
        assert not bits & mdg.STATUS_BOUNDS, f"{what}: MDG_STATUS_BOUNDS"
        seen.append(what)

    swarms = {"full_aero": wl.full_aero(81, n_envs=2048), "uneven": wl.uneven(82, n_envs=1024),
              "dense": wl.dense(83, n_envs=64), "single": wl.single(84, n_envs=256)}
    for name, sw in swarms.items():
        h = mdg.Handle(sw.drones_per_env, sw.flags)
        h.set_action_types(sw.act_type)
        st = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
        act = torch.as_tensor(wl.mixed_actions(sw, 85, 0, hover), device=dev)
        kin, idx, rel = h.new_obs(dev)
        for block in sorted({h.block_size, 32 * ((max(sw.drones_per_env) + 31) // 32), 256, 1024}):
            if block < max(sw.drones_per_env):
                continue
            h.set_block_size(block)
            h.step(st, act, mdg.ACT_MIXED, 5)
            h.step_obs(st, act, mdg.ACT_MIXED, 5, kin, idx, rel)
            check(h, f"{name} step/step_obs block {block}")
            acts = torch.as_tensor(np.stack([wl.mixed_actions(sw, 86, k, hover) for k in range(3)]), device=dev)
            kin3 = torch.empty((3,) + tuple(kin.shape), device=dev)
            idx3 = torch.empty((3,) + tuple(idx.shape), dtype=torch.int32, device=dev)
            rel3 = torch.empty((3,) + tuple(rel.shape), device=dev)
            h.rollout(st, acts, mdg.ACT_MIXED, 5, 3, mdg.OBS_EVERY_STEP, kin3, idx3, rel3)
            check(h, f"{name} rollout block {block}")
        h.obs(st, kin, idx, rel)
        frames = h.new_frames(dev)
        h.render(st, *frames)
        check(h, f"{name} render")
        rpm = torch.empty((sw.n, 4), device=dev)
        h.pid(st, torch.as_tensor(wl.waypoints(87, sw.n), device=dev), rpm)
        check(h, f"{name} obs/pid")
        if min(sw.drones_per_env) == max(sw.drones_per_env) and sw.drones_per_env[0] <= 32:
            raw = torch.empty((sw.n, mdg.MLP_IN), device=dev)
            h.features(st, rpm, raw)
            m = mdg.MLP((sw.n + 127) // 128 * 128, wl.mlp_init(88))
            z = np.zeros(mdg.MLP_IN, np.float32)
            m.set_normalization(z, np.ones(mdg.MLP_IN, np.float32), np.zeros(mdg.MLP_OUT, np.float32),
                                np.ones(mdg.MLP_OUT, np.float32), z - 1e30, z + 1e30)
            nfb = torch.zeros(1, dtype=torch.int32, device=dev)
            m.step(h, st, act, mdg.ACT_MIXED, 5, 1e30, nfb)   # every environment on the network
            m.step(h, st, act, mdg.ACT_MIXED, 5, 0.0, nfb)    # every environment on the fallback
            torch.cuda.synchronize()
            assert int(nfb) == sw.n_envs
            check(h, f"{name} surrogate")
    # the RK4 and per-rotor ground-height variants (runtime flags and sizes; the small-block
    # and any-size kernels)
    rk4 = mdg.Constants.cf2x()
    rk4.integrator = mdg.INTEGRATOR_RK4
    gnd_rotor = mdg.Constants.cf2p()
    gnd_rotor.gnd_heights = mdg.GND_ROTOR
    cf2x = mdg.Constants.cf2x()
    for name, c, tag in (("uneven", rk4, "rk4"), ("dense", rk4, "rk4"), ("uneven", gnd_rotor, "per-rotor"),
                         ("uneven", cf2x, "all action types")):
        sw = swarms[name]
        h = mdg.Handle(sw.drones_per_env, sw.flags, c)
        if tag == "all action types":
            types = wl.all_action_types(91, sw.n_envs)
            h.set_action_types(types)
            act = torch.as_tensor(wl.typed_actions(sw.drones_per_env, types, 92, 0, hover, 0.265), device=dev)
        else:
            h.set_action_types(sw.act_type)
            act = torch.as_tensor(wl.mixed_actions(sw, 90, 0, hover), device=dev)
        st = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
        kin, idx, rel = h.new_obs(dev)
        for block in sorted({h.block_size, 256, 1024}):
            if block < max(sw.drones_per_env):
                continue
            h.set_block_size(block)
            h.step_obs(st, act, mdg.ACT_MIXED, 5, kin, idx, rel)
            h.rollout(st, act[None], mdg.ACT_MIXED, 5, 1)
            check(h, f"{name} {tag} block {block}")
    # the randomization variants (uneven tables and any-size blocks)
    for name in ("uneven", "dense"):
        sw = swarms[name]
        h = mdg.Handle(sw.drones_per_env, sw.flags)
        h.set_action_types(sw.act_type)
        motor, hist, wind = h.new_randomization_state(3, dev)
        h.set_randomization(torch.as_tensor(wl.dr_table(93, sw.n_envs, depth=3), device=dev), motor, hist, wind, 5)
        st = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
        act = torch.as_tensor(wl.mixed_actions(sw, 94, 0, hover), device=dev)
        kin, idx, rel = h.new_obs(dev)
        for block in sorted({h.block_size, 256, 1024}):
            if block < max(sw.drones_per_env):
                continue
            h.set_block_size(block)
            h.step_obs(st, act, mdg.ACT_MIXED, 5, kin, idx, rel)
            h.rollout(st, act[None], mdg.ACT_MIXED, 5, 1)
            check(h, f"{name} randomized block {block}")
    # the allocation-free entry point builds its tables in static scratch
    sw = swarms["uneven"]
    st = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
    act = torch.as_tensor(wl.mixed_actions(sw, 89, 0, hover), device=dev)
    kin = torch.empty((sw.n, mdg.KIN_DIM), device=dev)
    idx = torch.empty((sw.n, mdg.NBR_K), dtype=torch.int32, device=dev)
    rel = torch.empty((sw.n, mdg.NBR_K * mdg.NBR_FEAT), device=dev)
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    VP = ctypes.c_void_p
    dpe = np.ascontiguousarray(sw.drones_per_env, np.int32)
    flg = np.ascontiguousarray(sw.flags, np.uint32)
    at = np.ascontiguousarray(sw.act_type, np.uint8)
    rc = mdg.lib().mdg_step_obs_noalloc(None, sw.n_envs, dpe.ctypes.data_as(VP), flg.ctypes.data_as(VP),
                                        at.ctypes.data_as(VP), VP(st.data_ptr()), VP(act.data_ptr()), mdg.ACT_MIXED, 5,
                                        VP(kin.data_ptr()), VP(idx.data_ptr()), VP(rel.data_ptr()),
                                        VP(status.data_ptr()), VP(torch.cuda.current_stream().cuda_stream))
    assert rc == mdg.OK, mdg.lib().mdg_last_error()
    torch.cuda.synchronize()
    assert not int(status[0].item()) & mdg.STATUS_BOUNDS, "noalloc: MDG_STATUS_BOUNDS"
    print(len(seen) + 1, "checked launches;", "all checks passed")


if __name__ == "__main__" and "--run" in sys.argv:
    _run()
