"""GPU parity of the camera frames (mdg_render) against the oracle's ray caster.

Every pixel the oracle does not mark ambiguous (oracle.camera.ambiguous: a decision within
the relative margin a float32 ray caster may flip) must have the oracle's segment id
exactly, its depth within 1e-5 relative (+inf for sky on both sides; a ground hit's depth
-o_z / d_z amplifies a float32 error of the ray direction by 1/|d_z|, so ground pixels take
1e-5 + 1e-6 / |d_z|; a ray-ellipsoid hit's depth amplifies the error of its discriminant by
about 1/(2 sqrt(m)), m = |disc| / B^2 its grazing margin, so drone pixels take
1e-5 + 1e-6 / sqrt(m)) and its RGB within one step per channel (round(255 c) of a float and
a double shade); an ambiguous pixel must
carry one of the ids it could show (sky, ground or a drone of its environment).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import camera
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import oracle_arrays

pytestmark = pytest.mark.gpu
P = oracle.cf2x()


def _check(h, x, dpe, rgba, depth, seg, cams=None, what=""):
    env_off = np.concatenate([[0], np.cumsum(dpe)])
    rgba, depth, seg = rgba.cpu().numpy(), depth.cpu().numpy(), seg.cpu().numpy()
    env_of = np.repeat(np.arange(len(dpe)), dpe)
    cams = range(x.shape[0]) if cams is None else cams
    n_px = n_amb = 0
    for g in cams:
        e = env_of[g]
        b, N = int(env_off[e]), int(dpe[e])
        ro, zo, so, m = camera.render(P, x[b:b + N], g - b, first_index=b)
        amb = camera.ambiguous(m)
        ok = ~amb
        n_px += ok.size
        n_amb += int(amb.sum())
        tag = f"{what} camera {g}"
        np.testing.assert_array_equal(seg[g][ok], so[ok], err_msg=tag)
        zg, zr = depth[g][ok].astype(np.float64), zo[ok]
        assert np.array_equal(np.isinf(zg), np.isinf(zr)), tag
        fin = np.isfinite(zr)
        rtol = 1e-5 + np.where(so[ok] == 0, 1e-6 / np.maximum(m["horizon"][ok], 1e-12),
                               np.where(so[ok] > 0, 1e-6 / np.sqrt(np.maximum(m["grazing"][ok], 1e-12)), 0.0))
        rel = np.abs(zg[fin] - zr[fin]) / np.abs(zr[fin])
        assert np.all(rel <= rtol[fin]), f"{tag}: depth off by {np.max(rel / rtol[fin]):.3g} x the tolerance"
        diff = np.abs(rgba[g][ok].astype(int) - ro[ok].astype(int))
        assert diff.max(initial=0) <= 1, f"{tag}: rgb off by {diff.max()}"
        assert np.all(rgba[g][..., 3] == 255)
        valid = {-1, 0} | set(range(1 + b, 1 + b + N)) - {1 + g}
        assert set(np.unique(seg[g][amb])) <= valid, tag
    assert n_amb <= 0.01 * n_px, f"{what}: {n_amb} ambiguous pixels of {n_px}"


@pytest.mark.parametrize("recipe", ["full_aero", "uneven", "dense", "tumbling"])
def test_frames_match_oracle(cuda, recipe):
    if recipe == "full_aero":
        sw = wl.full_aero(101, n_envs=48)
    elif recipe == "uneven":
        sw = wl.uneven(102, n_envs=24)
    elif recipe == "dense":
        sw = wl.dense(103, n_envs=2)
    else:  # arbitrary attitudes: cameras looking up, sideways, upside down
        sw = wl.full_aero(104, n_envs=48)
        p, q, v, w = wl.random_states(104, sw.n)
        sw.q = q
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    rgba, depth, seg = h.new_frames(cuda)
    h.render(state, rgba, depth, seg)
    torch.cuda.synchronize()
    x, _, _ = oracle_arrays(state)
    cams = None if sw.n <= 256 else np.random.default_rng(0).choice(sw.n, 256, replace=False)
    _check(h, x, sw.drones_per_env, rgba, depth, seg, cams, recipe)
    assert h.status()[0] == mdg.OK


def test_full_size_frames_on_sampled_cameras(cuda):
    """The full-aero swarm at its benchmark size (16384 envs x 4 drones): 64 sampled cameras."""
    sw = wl.full_aero(1)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    rgba, depth, seg = h.new_frames(cuda)
    h.render(state, rgba, depth, seg)
    torch.cuda.synchronize()
    x, _, _ = oracle_arrays(state)
    cams = np.random.default_rng(1).choice(sw.n, 64, replace=False)
    _check(h, x, sw.drones_per_env, rgba, depth, seg, cams, "full size")


def test_optional_outputs_and_arguments(cuda):
    sw = wl.uneven(105, n_envs=16)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    rgba, depth, seg = h.new_frames(cuda)
    h.render(state, rgba, depth, seg)
    _, _, seg2 = h.new_frames(cuda, rgba=False, depth=False)
    h.render(state, seg=seg2)
    rgba3, _, _ = h.new_frames(cuda, depth=False, seg=False)
    h.render(state, rgba=rgba3)
    torch.cuda.synchronize()
    assert torch.equal(seg, seg2) and torch.equal(rgba, rgba3)
    L = mdg.lib()
    assert L.mdg_render(h._h, state.data_ptr(), rgba.data_ptr() + 1, None, None, None) == mdg.ERR_ARG
