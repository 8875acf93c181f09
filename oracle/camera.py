"""FP64 reference of the headless camera observation (test infrastructure only).

TEST INFRASTRUCTURE ONLY: used by the test suite, never by the library.

Section 3.4.4 (Observation types): RGB frames (48, 64, 4) uint8 from each drone's onboard
camera with a 60 degree field of view, at [0.02, 0, 0] in the body frame. The paper renders
them with MuJoCo's OpenGL renderer and the Crazyflie meshes; neither exists here, so the
frames are ray cast from primitive shapes. Readings (none of this is printed):
  - pinhole camera looking along body +x, image right = body -y, image up = body +z;
    60 degrees is the vertical field of view (MuJoCo's fovy); pixel (r, c) looks through
    the centre of its cell, row 0 at the top;
  - the scene: every other drone of the environment as an oblate ellipsoid in its own body
    frame with semi-axes (L + r_p, L + r_p, 0.3 (L + r_p)); the ground plane z = 0 with a
    0.5 m checkerboard, seen from above only; the camera's own drone is not drawn;
  - colours: ground squares 0.55 / 0.35 grey, drone k (global index) the palette entry
    k mod 8, each shaded by ambient 0.35 + diffuse 0.65 max(0, n . l) with the unit light
    direction l along (0.3, 0.2, 1.0); sky (0.55, 0.70, 0.90) unshaded; channel value
    round(255 c), alpha 255;
  - depth: distance along the optical axis (z-depth) to the nearest hit at t > 1e-4 m along
    the ray, +inf where no surface is hit;
  - segmentation: -1 sky, 0 ground, 1 + the global index of the drone hit.
render() also returns, per pixel, the margins of the decisions it depends on, each as
the relative change of the inputs that would flip it: "grazing" (|disc| / B^2 of the
nearest ellipsoid the ray passes: how far it is from the silhouette), "gap" (the relative
distance between the nearest and the second-nearest surface), "edge" (a ground hit point's
distance to a checker edge over t (1 + 1/|d_z|), the distance a relative error of the ray
moves it), "horizon" (|d_z| of a ray that could hit the ground). A pixel with a small
margin may legitimately render either way in finite precision.
"""
from __future__ import annotations

import numpy as np

from . import rotation

H, W = 48, 64
FOVY_DEG = 60.0
CAM_POS = np.array([0.02, 0.0, 0.0])
T_MIN = 1e-4
CHECKER = 0.5
GROUND = np.array([[0.55, 0.55, 0.55], [0.35, 0.35, 0.35]])
SKY = np.array([0.55, 0.70, 0.90])
PALETTE = np.array([[0.90, 0.25, 0.20], [0.20, 0.70, 0.30], [0.20, 0.35, 0.90], [0.95, 0.75, 0.15],
                    [0.70, 0.30, 0.80], [0.15, 0.75, 0.80], [0.95, 0.50, 0.20], [0.60, 0.60, 0.65]])
LIGHT = np.array([0.3, 0.2, 1.0]) / np.linalg.norm([0.3, 0.2, 1.0])
AMBIENT, DIFFUSE = 0.35, 0.65


def semi_axes(P):
    a = P.arm + P.prop_radius
    return np.array([a, a, 0.3 * a])


def pixel_rays_body():
    """[H, W, 3] unnormalized body-frame ray directions (forward component 1)."""
    th = np.tan(np.radians(FOVY_DEG) / 2)
    c = (np.arange(W) + 0.5) / W * 2 - 1
    r = 1 - (np.arange(H) + 0.5) / H * 2
    nx = c * th * W / H
    ny = r * th
    d = np.zeros((H, W, 3))
    d[..., 0] = 1.0
    d[..., 1] = -nx[None, :]
    d[..., 2] = ny[:, None]
    return d


def _shade(base, n):
    return base * (AMBIENT + DIFFUSE * np.maximum(0.0, n @ LIGHT))[..., None]


def render(P, x_env, j, first_index=0):
    """The frame of drone j of one environment (x_env [N, 13] float64 states; global index
    of drone k = first_index + k). Returns (rgba [H, W, 4] uint8, depth [H, W] float64,
    seg [H, W] int32, margins: dict of [H, W] float64 "grazing", "gap", "edge", "horizon")."""
    x_env = np.asarray(x_env, np.float64)
    Rj = rotation(x_env[j, 3:7])
    o = x_env[j, 0:3] + Rj @ CAM_POS
    db = pixel_rays_body()
    fwd = Rj[:, 0]
    d = db @ Rj.T                                  # world directions, forward component 1 in the camera
    dn = d / np.linalg.norm(d, axis=-1, keepdims=True)
    t_best = np.full((H, W), np.inf)
    seg = np.full((H, W), -1, np.int32)
    color = np.broadcast_to(SKY, (H, W, 3)).copy()
    inf = np.full((H, W), np.inf)
    margins = {"grazing": inf.copy(), "gap": inf.copy(), "edge": inf.copy(), "horizon": inf.copy()}
    t_all = []
    # ground plane, from above
    if o[2] > 0:
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(dn[..., 2] < 0, -o[2] / dn[..., 2], np.inf)
        t = np.where(t > T_MIN, t, np.inf)
        hit = np.isfinite(t)
        pt = o + np.where(hit, t, 0.0)[..., None] * dn
        gx, gy = pt[..., 0] / CHECKER, pt[..., 1] / CHECKER
        par = np.mod(np.floor(gx) + np.floor(gy), 2).astype(int)
        col = _shade(GROUND[par], np.broadcast_to(np.array([0.0, 0.0, 1.0]), (H, W, 3)))
        # margins: a ray near the horizon; a hit point near a checker edge, as the relative
        # change of the ray that moves the hit point onto the edge (a relative error e in the
        # ray moves the hit point by about e t (1 + 1/|dz|))
        fx, fy = np.abs(gx - np.round(gx)), np.abs(gy - np.round(gy))
        reach = np.where(hit, t, 1.0) * (1.0 + 1.0 / np.maximum(np.abs(dn[..., 2]), 1e-30))
        margins["edge"] = np.where(hit, CHECKER * np.minimum(fx, fy) / reach, np.inf)
        margins["horizon"] = np.abs(dn[..., 2])
        t_all.append(t)
        better = t < t_best
        t_best = np.where(better, t, t_best)
        seg = np.where(better, 0, seg)
        color = np.where(better[..., None], col, color)
    # the other drones
    s = semi_axes(P)
    for k in range(x_env.shape[0]):
        if k == j:
            continue
        Rk = rotation(x_env[k, 3:7])
        O = (Rk.T @ (o - x_env[k, 0:3])) / s
        D = (dn @ Rk) / s
        A = np.sum(D * D, axis=-1)
        B = 2 * (D @ O)
        C = O @ O - 1
        disc = B * B - 4 * A * C
        sq = np.sqrt(np.maximum(disc, 0.0))
        t1 = (-B - sq) / (2 * A)
        t2 = (-B + sq) / (2 * A)
        t = np.where(disc >= 0, np.where(t1 > T_MIN, t1, np.where(t2 > T_MIN, t2, np.inf)), np.inf)
        # margin: how far the ray is from grazing the ellipsoid, relative
        margins["grazing"] = np.minimum(margins["grazing"], np.abs(disc) / np.maximum(B * B, 1e-30))
        pb = O + np.where(np.isfinite(t), t, 0.0)[..., None] * D  # hit point, scaled body frame
        nb = pb / s                                # gradient of |p/s|^2 in the body frame
        n = nb @ Rk.T
        n = n / np.maximum(np.linalg.norm(n, axis=-1, keepdims=True), 1e-30)
        col = _shade(PALETTE[(first_index + k) % len(PALETTE)], n)
        t_all.append(t)
        better = t < t_best
        t_best = np.where(better, t, t_best)
        seg = np.where(better, 1 + first_index + k, seg)
        color = np.where(better[..., None], col, color)
    # margin: the gap between the nearest and the second-nearest surface
    if len(t_all) > 1:
        ts = np.sort(np.stack(t_all), axis=0)
        fin = np.isfinite(ts[1])
        gap = np.where(fin, (np.where(fin, ts[1], 1.0) - np.where(fin, ts[0], 0.0)) / np.where(fin, ts[1], 1.0), np.inf)
        margins["gap"] = gap
    depth = np.where(np.isfinite(t_best), t_best * (dn @ fwd), np.inf)
    rgba = np.empty((H, W, 4), np.uint8)
    rgba[..., 0:3] = np.round(255 * np.clip(color, 0, 1)).astype(np.uint8)
    rgba[..., 3] = 255
    return rgba, depth, seg, margins


def ambiguous(margins, grazing=1e-4, gap=1e-5, edge=1e-6, horizon=1e-6):
    """Pixels whose render may flip in single precision: any margin under its threshold (the
    relative errors a float32 ray caster makes in each decision, with room to spare)."""
    return ((margins["grazing"] < grazing) | (margins["gap"] < gap) | (margins["edge"] < edge) |
            (margins["horizon"] < horizon))
