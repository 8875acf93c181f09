"""Roll, pitch and yaw of the KIN observation against float64 mathematics.

The kernels compute the angles with their own arctangent (an octant reduction and a
fitted polynomial) and arcsine (through the arctangent); this checks them through the
product path (mdg_obs) on a million seeded attitudes plus exact special cases. The
reference is numpy's float64 arctan2 / arcsin of the float32 quaternion, so the bound
has two parts: the functions' own error (a few 1e-7 rad) and the float32 rounding of their
arguments (~3e-7 absolute), amplified by the conditioning of the angle: 1/r for the
arctangents (r the length of the argument pair, cos(pitch)) and 1/sqrt(1 - s^2) for the
arcsine. Near gimbal lock (r < 1e-3) only the range is checked.
"""
import numpy as np
import pytest
import torch

import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FN_ERR = 4e-7     # the arctangent's polynomial, reciprocal and octant steps
ARG_ERR = 4e-7    # float32 rounding of each argument (sums of three products of |.| <= 1)


def _wrap(d):
    return (d + np.pi) % (2.0 * np.pi) - np.pi


def _quaternions(n, seed=3):
    idx = np.arange(n, dtype=np.uint64)[:, None]
    q = wl.uniform_range(-1.0, 1.0, seed, 40, 0, idx, np.arange(4, dtype=np.uint64)[None, :]).astype(np.float64)
    norm = np.linalg.norm(q, axis=1)
    q = q[norm > 0.1] / norm[norm > 0.1, None]
    s = np.sqrt(0.5)
    special = np.array([
        [1, 0, 0, 0], [-1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1], [0, 0, 0, -1],
        [s, s, 0, 0], [s, -s, 0, 0], [s, 0, 0, s], [s, 0, 0, -s], [s, 0, s, 0], [s, 0, -s, 0],
        [np.cos(1e-4), np.sin(1e-4), 0, 0], [np.cos(1e-4), 0, 0, -np.sin(1e-4)],
        [np.cos(1.5), 0, 0, np.sin(1.5)], [np.cos(1.5), np.sin(1.5), 0, 0],
        [1e-20, 0, 0, 1], [0, 1e-20, 0, 1], [0, 0, 1e-20, 1],
    ], dtype=np.float64)
    special /= np.linalg.norm(special, axis=1, keepdims=True)
    return np.concatenate([special, q]).astype(np.float32)


def test_rpy_against_float64(cuda):
    q32 = _quaternions(1 << 20)
    n = q32.shape[0]
    h = mdg.Handle(np.ones(n, np.int32), np.zeros(n, np.uint32))
    z = np.zeros((n, 3), np.float32)
    state = mdg.pack_state(z, q32, z, z, device=cuda)
    kin, idx, rel = h.new_obs(cuda)
    h.obs(state, kin, idx, rel)
    torch.cuda.synchronize()
    assert h.status()[0] == mdg.OK
    rpy = kin[:, 7:10].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(kin[:, 3:7].cpu().numpy(), q32)  # the quaternion passes through

    w, x, y, zq = (q32[:, k].astype(np.float64) for k in range(4))
    args = [(2 * (w * x + y * zq), 1 - 2 * (x * x + y * y)), (2 * (w * zq + x * y), 1 - 2 * (y * y + zq * zq))]
    s = np.clip(2 * (w * y - zq * x), -1.0, 1.0)
    c = np.sqrt((1 - s) * (1 + s))
    assert np.all(np.isfinite(rpy))
    assert np.all(np.abs(rpy[:, [0, 2]]) <= np.float32(np.pi)) and np.all(np.abs(rpy[:, 1]) <= np.float32(np.pi / 2))
    ok = c > 1e-3
    for col, (ya, xa) in zip((0, 2), args):
        ref = np.arctan2(ya, xa)
        r = np.hypot(ya, xa)
        err = np.abs(_wrap(rpy[:, col] - ref))
        bound = FN_ERR + ARG_ERR / np.maximum(r, 1e-300)
        bad = ok & (err > bound)
        assert not bad.any(), f"angle {col}: {int(bad.sum())} outside the bound, worst {err[ok].max():.3g}"
    err = np.abs(rpy[:, 1] - np.arcsin(s))
    bound = FN_ERR + ARG_ERR / np.maximum(c, 1e-300)
    bad = ok & (err > bound)
    assert not bad.any(), f"pitch: {int(bad.sum())} outside the bound, worst {err[ok].max():.3g}"
    # no systematic offset: the typical error is a fraction of the bound
    well = ok & (c > 0.5)
    assert np.median(np.abs(rpy[well, 1] - np.arcsin(s[well]))) < 1.5e-7


def test_rpy_special_cases_exact(cuda):
    """Attitudes whose angles are exact in float32 come out exact, signs of pi included."""
    q = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)
    expect = np.array([[0, 0, 0], [0, 0, np.pi], [np.pi, 0, 0], [np.pi, 0, np.pi]], np.float32)
    n = q.shape[0]
    h = mdg.Handle(np.ones(n, np.int32), np.zeros(n, np.uint32))
    z = np.zeros((n, 3), np.float32)
    state = mdg.pack_state(z, q, z, z, device=cuda)
    kin, idx, rel = h.new_obs(cuda)
    h.obs(state, kin, idx, rel)
    torch.cuda.synchronize()
    got = kin[:, 7:10].cpu().numpy()
    # identity: all zero; yaw of pi about z: +pi (the arguments are (+0, -1))
    np.testing.assert_array_equal(got[0], expect[0])
    np.testing.assert_allclose(got[1], expect[1], atol=4e-7, rtol=0)
    # a half turn about x (or y) reads as roll pi (and yaw pi) with pitch 0, up to the sign of pi
    np.testing.assert_allclose(np.abs(got[2:]), expect[2:], atol=4e-7, rtol=0)
