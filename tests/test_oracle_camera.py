"""Pins of the oracle's camera (CPU): closed forms for the ground seen from a level camera,
sky above the horizon, exact colours, translation and mirror symmetry, invariance of depth
and segmentation under a yaw of the whole scene about the camera's vertical axis, the
segmentation ids, and a small share of ambiguous pixels in random scenes."""
import numpy as np
import pytest

import oracle
from oracle import camera

P = oracle.cf2x()
TH = np.tan(np.radians(camera.FOVY_DEG) / 2)


def _x(p, yaw=0.0):
    return np.array([*p, np.cos(yaw / 2), 0.0, 0.0, np.sin(yaw / 2), 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])


def test_level_camera_ground_and_sky():
    """Alone at height h, level: row r below the horizon sees the ground at z-depth h / (-n_y)
    (the ray's forward component is 1), rows above see the sky."""
    h = 1.3
    rgba, depth, seg, _ = camera.render(P, _x((0.1, -0.2, h))[None], 0)
    ny = (1 - (np.arange(camera.H) + 0.5) / camera.H * 2) * TH
    lower = ny < 0
    np.testing.assert_allclose(depth[lower], np.repeat((h / (-ny[lower]))[:, None], camera.W, axis=1), rtol=1e-12)
    assert np.all(seg[lower] == 0) and np.all(seg[~lower] == -1)
    assert np.all(np.isinf(depth[~lower]))
    sky = np.round(255 * camera.SKY).astype(np.uint8)
    assert np.all(rgba[~lower][..., 0:3] == sky) and np.all(rgba[..., 3] == 255)
    shade = camera.AMBIENT + camera.DIFFUSE * camera.LIGHT[2]
    greys = {int(np.round(255 * g * shade)) for g in camera.GROUND[:, 0]}
    assert set(np.unique(rgba[lower][..., 0])) == greys


def test_camera_below_ground_sees_no_ground():
    rgba, depth, seg, _ = camera.render(P, _x((0.0, 0.0, -0.5))[None], 0)
    assert np.all(seg == -1)


def test_drone_ahead_depth_bound_and_horizontal_translation():
    """A drone ahead on the optical axis at distance D: no pixel sees it nearer than its front
    surface, D - 0.02 - a, and the nearest is within 2 cm of it; its segment id is 1
    + its global index; nearer, it covers more pixels. Translating the whole scene
    horizontally changes neither depth nor segmentation (the ground plane is invariant)."""
    h = 2.0
    a = camera.semi_axes(P)[0]
    cam = _x((0.0, 0.0, h))
    counts = []
    for D in (0.4, 0.9):
        x = np.stack([cam, _x((D, 0.0, h))])
        _, z, s, m = camera.render(P, x, 0, first_index=10)
        mine = s == 12
        assert mine.any() and set(np.unique(s)) <= {-1, 0, 12}
        assert z[mine].min() >= D - 0.02 - a - 1e-12
        assert z[mine].min() <= D - 0.02 - a + 0.02  # the nearest rays pass 0.012 rad off the axis
        counts.append(mine.sum())
        shift = np.array([3.7, -1.2, 0.0])
        xs = x.copy()
        xs[:, 0:3] += shift
        _, z2, s2, m2 = camera.render(P, xs, 0, first_index=10)
        ok = ~camera.ambiguous(m) & ~camera.ambiguous(m2)
        np.testing.assert_array_equal(s[ok], s2[ok])
        np.testing.assert_allclose(z[ok], z2[ok], rtol=1e-9)
    assert counts[0] > counts[1]


def test_mirror_symmetry():
    h = 1.0
    cam = _x((0.0, 0.0, h))
    _, za, sa, _ = camera.render(P, np.stack([cam, _x((0.8, 0.15, h + 0.02))]), 0)
    _, zb, sb, _ = camera.render(P, np.stack([cam, _x((0.8, -0.15, h + 0.02))]), 0)
    np.testing.assert_array_equal(sa, sb[:, ::-1])
    np.testing.assert_allclose(za, zb[:, ::-1], rtol=1e-12)


def test_yaw_of_the_scene_about_the_camera_axis():
    """Rotating every drone (position about the camera's vertical axis, and orientation) by
    the same yaw changes neither depth nor segmentation (only the checker colours move)."""
    rng = np.random.default_rng(3)
    base = [_x((0.0, 0.0, 1.0), 0.0)] + [_x((rng.uniform(0.5, 2), rng.uniform(-0.6, 0.6), rng.uniform(0.8, 1.2)),
                                          rng.uniform(-1, 1)) for _ in range(3)]
    x0 = np.stack(base)
    psi = 0.9
    Rz = np.array([[np.cos(psi), -np.sin(psi), 0], [np.sin(psi), np.cos(psi), 0], [0, 0, 1]])
    x1 = x0.copy()
    for k in range(4):
        x1[k, 0:2] = (Rz @ (x0[k, 0:3] - x0[0, 0:3]))[0:2] + x0[0, 0:2]
        x1[k, 3:7] = oracle.quat_mul([np.cos(psi / 2), 0, 0, np.sin(psi / 2)], x0[k, 3:7])
    _, za, sa, ma = camera.render(P, x0, 0)
    _, zb, sb, mb = camera.render(P, x1, 0)
    ok = ~camera.ambiguous(ma) & ~camera.ambiguous(mb)
    np.testing.assert_array_equal(sa[ok], sb[ok])
    np.testing.assert_allclose(za[ok], zb[ok], rtol=1e-9)
    assert len(set(np.unique(sa)) - {-1, 0}) >= 1


def test_ambiguous_pixels_are_rare():
    rng = np.random.default_rng(4)
    n_amb, n_px = 0, 0
    for _ in range(10):
        x = np.stack([_x((rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.3, 2)), rng.uniform(-3, 3))
                      for _ in range(6)])
        for j in range(6):
            _, _, seg, m = camera.render(P, x, j)
            n_amb += int(camera.ambiguous(m).sum())
            n_px += seg.size
    assert n_amb / n_px < 0.005, n_amb / n_px


def test_checker_seen_by_a_level_camera():
    """The ground's checker parity under a level camera at (x0, y0, h) equals the parity of
    the hit points of the pinhole model: pixel (r, c) looks along (1, -n_x, n_y) with
    n_x = ((c + 0.5)/W 2 - 1) tan(30 deg) W/H and n_y = (1 - (r + 0.5)/H 2) tan(30 deg), and
    hits the ground at (x0 + 0.02 + h/(-n_y), y0 - n_x h/(-n_y)). Away from the horizon and
    the checker edges."""
    x0, y0, h = 0.13, -0.31, 0.9
    rgba, _, seg, m = camera.render(P, _x((x0, y0, h))[None], 0)
    r = np.arange(camera.H)[:, None]
    c = np.arange(camera.W)[None, :]
    nx = ((c + 0.5) / camera.W * 2 - 1) * TH * camera.W / camera.H
    ny = (1 - (r + 0.5) / camera.H * 2) * TH
    below = np.broadcast_to(ny < -0.05, (camera.H, camera.W))
    t = h / np.where(ny < 0, -ny, 1.0)
    gx, gy = (x0 + 0.02 + t) / camera.CHECKER, (y0 - nx * t) / camera.CHECKER
    parity = np.mod(np.floor(gx) + np.floor(gy), 2).astype(int)
    shade = camera.AMBIENT + camera.DIFFUSE * camera.LIGHT[2]
    expect = np.round(255 * camera.GROUND[parity, 0] * shade)
    ok = below & ~camera.ambiguous(m)
    assert ok.sum() > 500
    np.testing.assert_array_equal(rgba[..., 0][ok], expect[ok])
