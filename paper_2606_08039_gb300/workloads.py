"""Seeded synthetic workloads: initial swarms, per-environment physics subsets and actions.

This module only draws inputs; it holds none of the simulator's arithmetic. The tests
feed the same arrays to the CUDA library and to the FP64 oracle, and the benchmark uses
them for its timed runs. Every value is rounded to float32 (the precision the library
consumes) before either side sees it.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) chained over
(seed, stream, step, index, component), the top 24 bits giving a uniform float in [0, 1)
that float32 represents exactly. The draw for any drone, step and component can thus be
recomputed on its own.

Recipes (the paper fixes f_sim = 240 Hz and f_ctrl = 48 Hz, 5 substeps per control step;
the swarm shapes are the five benchmark configurations of this project):
  single     64 envs x 1 drone, ground effect + drag; x, y ~ U[-1, 1] m, z ~ U[0.05, 1] m,
             roll/pitch/yaw ~ U[-0.2, 0.2] rad, zero velocity and body rate; RPM actions
             U[0.9, 1.1] x HOVER_RPM per motor, redrawn every control step; 240 control steps.
  full_aero  16384 envs x 4 drones, ground effect + drag + downwash; a 2 x 2 grid of 0.3 m
             spacing centred at (0, 0, 1) m with U[-0.05, 0.05] m jitter per axis, level, at
             rest; PID waypoints U[-2, 2]^2 x U[0.2, 2] m, yaw 0, fixed for the episode;
             1000 control steps; KIN + 4-neighbour observations.
  uneven     4096 envs with N drawn uniformly from {1, 2, 4, 8, 16, 32}; physics subset drawn
             uniformly from the 8 combinations of {ground, drag, downwash}; action type RPM or
             PID drawn per env; drones on a cubic 0.3 m lattice of ceil(N^(1/3)) per side
             whose lowest layer is at z = 1 m, U[-0.05, 0.05] m jitter; 32 control steps.
  dense      1024 envs x 64 drones, full aero; a 4 x 4 x 4 lattice of 0.25 m spacing, lowest
             layer at z = 0.5 m, U[-0.03, 0.03] m jitter; RPM actions U[0.9, 1.1] x HOVER_RPM
             per motor per control step; 500 control steps.
  surrogate  evaluation swarm of 65536 envs x 4 drones with the full_aero initial distribution.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GND, DRAG, DW = 1, 2, 4
ACT_RPM, ACT_PID = 0, 1
ACT_RPM_NORM, ACT_ONE_D_RPM, ACT_VEL, ACT_ATTITUDE = 3, 4, 5, 6
ALL_ACTION_TYPES = (ACT_RPM, ACT_PID, ACT_RPM_NORM, ACT_ONE_D_RPM, ACT_VEL, ACT_ATTITUDE)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# generator streams
S_POS, S_ATT, S_ACT, S_WAYPOINT, S_ENV_N, S_ENV_FLAGS, S_ENV_ACT, S_VEL = 1, 2, 3, 4, 5, 6, 7, 8


def splitmix64(x) -> np.ndarray:
    """One SplitMix64 output for each 64-bit input (vectorised, wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, step, index, comp) -> np.ndarray:
    """U[0, 1) as float32 for the broadcast counters (seed, stream, step, index, comp)."""
    h = splitmix64(np.uint64(seed))
    for field in (stream, step, index, comp):
        h = splitmix64(h ^ np.asarray(field, dtype=np.uint64))
    return ((h >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))).astype(np.float32)


def uniform_range(lo, hi, seed, stream, step, index, comp) -> np.ndarray:
    u = uniform(seed, stream, step, index, comp).astype(np.float64)
    return (lo + (hi - lo) * u).astype(np.float32)


def quat_from_rpy(rpy: np.ndarray) -> np.ndarray:
    """[w, x, y, z] of the ZYX rotation Rz(yaw) Ry(pitch) Rx(roll), float32."""
    r, p, y = (rpy[..., i].astype(np.float64) / 2 for i in range(3))
    cr, sr, cp, sp, cy, sy = np.cos(r), np.sin(r), np.cos(p), np.sin(p), np.cos(y), np.sin(y)
    q = np.stack([cr * cp * cy + sr * sp * sy,
                  sr * cp * cy - cr * sp * sy,
                  cr * sp * cy + sr * cp * sy,
                  cr * cp * sy - sr * sp * cy], axis=-1)
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    return q.astype(np.float32)


@dataclasses.dataclass
class Swarm:
    """A batch of environments in CSR order (drones of env e are env_off[e] .. env_off[e+1]-1)."""
    drones_per_env: np.ndarray  # int32 [n_envs]
    flags: np.ndarray           # uint32 [n_envs] GND|DRAG|DW bits
    act_type: np.ndarray        # uint8 [n_envs] ACT_RPM / ACT_PID
    p: np.ndarray               # float32 [n, 3]
    q: np.ndarray               # float32 [n, 4]  (w, x, y, z)
    v: np.ndarray               # float32 [n, 3]
    w: np.ndarray               # float32 [n, 3]  body rates
    name: str = ""

    @property
    def n_envs(self) -> int:
        return int(self.drones_per_env.shape[0])

    @property
    def n(self) -> int:
        return int(self.p.shape[0])

    @property
    def env_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.drones_per_env, dtype=np.int64)]).astype(np.int32)

    def x13(self) -> np.ndarray:
        """[n, 13] = p, q, v, omega in float64 (exact copies of the float32 values)."""
        return np.concatenate([self.p, self.q, self.v, self.w], axis=1).astype(np.float64)

    def env_of_drone(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_envs, dtype=np.int32), self.drones_per_env)


def _lattice(N: int, side: int, spacing: float) -> np.ndarray:
    k = np.arange(N)
    return np.stack([k % side, (k // side) % side, k // (side * side)], axis=1).astype(np.float64) * spacing


def _jittered_lattice(seed, drones_per_env, spacing, z0, jitter, side_of) -> np.ndarray:
    env_off = np.concatenate([[0], np.cumsum(drones_per_env)])
    n = int(env_off[-1])
    p = np.zeros((n, 3))
    for N in np.unique(drones_per_env):
        side = side_of(int(N))
        base = _lattice(int(N), side, spacing)
        base[:, :2] -= (side - 1) * spacing / 2  # centred in x, y
        base[:, 2] += z0
        envs = np.nonzero(drones_per_env == N)[0]
        idx = (env_off[envs][:, None] + np.arange(N)[None, :]).reshape(-1)
        p[idx] = np.tile(base, (len(envs), 1))
    idx = np.arange(n, dtype=np.uint64)[:, None]
    p += uniform_range(-jitter, jitter, seed, S_POS, 0, idx, np.arange(3, dtype=np.uint64)[None, :])
    return p.astype(np.float32)


def _at_rest(n):
    q = np.zeros((n, 4), np.float32)
    q[:, 0] = 1
    return q, np.zeros((n, 3), np.float32), np.zeros((n, 3), np.float32)


def single(seed: int = 0, n_envs: int = 64) -> Swarm:
    idx = np.arange(n_envs, dtype=np.uint64)[:, None]
    lo = np.array([-1, -1, 0.05])
    hi = np.array([1, 1, 1.0])
    u = uniform(seed, S_POS, 0, idx, np.arange(3, dtype=np.uint64)[None, :]).astype(np.float64)
    p = (lo + (hi - lo) * u).astype(np.float32)
    rpy = uniform_range(-0.2, 0.2, seed, S_ATT, 0, idx, np.arange(3, dtype=np.uint64)[None, :])
    _, v, w = _at_rest(n_envs)
    return Swarm(np.ones(n_envs, np.int32), np.full(n_envs, GND | DRAG, np.uint32), np.zeros(n_envs, np.uint8),
                 p, quat_from_rpy(rpy), v, w, "single")


def full_aero(seed: int = 1, n_envs: int = 16384, drones: int = 4) -> Swarm:
    dpe = np.full(n_envs, drones, np.int32)
    p = _jittered_lattice(seed, dpe, 0.3, 1.0, 0.05, lambda N: max(1, math.ceil(math.sqrt(N))))
    q, v, w = _at_rest(p.shape[0])
    return Swarm(dpe, np.full(n_envs, GND | DRAG | DW, np.uint32), np.full(n_envs, ACT_PID, np.uint8),
                 p, q, v, w, "full_aero")


def uneven(seed: int = 2, n_envs: int = 4096, sizes=(1, 2, 4, 8, 16, 32)) -> Swarm:
    e = np.arange(n_envs, dtype=np.uint64)
    sizes = np.asarray(sizes, np.int32)
    dpe = sizes[np.minimum((uniform(seed, S_ENV_N, 0, e, 0) * len(sizes)).astype(np.int64), len(sizes) - 1)]
    flags = np.minimum((uniform(seed, S_ENV_FLAGS, 0, e, 0) * 8).astype(np.uint32), 7).astype(np.uint32)
    act = (uniform(seed, S_ENV_ACT, 0, e, 0) < 0.5).astype(np.uint8)
    p = _jittered_lattice(seed, dpe, 0.3, 1.0, 0.05, lambda N: max(1, math.ceil(round(N ** (1 / 3), 9))))
    q, v, w = _at_rest(p.shape[0])
    return Swarm(dpe, flags, act, p, q, v, w, "uneven")


def dense(seed: int = 5, n_envs: int = 1024) -> Swarm:
    dpe = np.full(n_envs, 64, np.int32)
    p = _jittered_lattice(seed, dpe, 0.25, 0.5, 0.03, lambda N: 4)
    q, v, w = _at_rest(p.shape[0])
    return Swarm(dpe, np.full(n_envs, GND | DRAG | DW, np.uint32), np.zeros(n_envs, np.uint8), p, q, v, w, "dense")


def surrogate_eval(seed: int = 4, n_envs: int = 65536) -> Swarm:
    s = full_aero(seed, n_envs)
    s.name = "surrogate_eval"
    return s


def rpm_actions(seed: int, n: int, step: int, hover_rpm: float, lo: float = 0.9, hi: float = 1.1) -> np.ndarray:
    """[n, 4] float32 RPMs U[lo, hi] x hover_rpm for one control step (hover_rpm is the caller's scale)."""
    u = uniform(seed, S_ACT, step, np.arange(n, dtype=np.uint64)[:, None], np.arange(4, dtype=np.uint64)[None, :])
    return (hover_rpm * (lo + (hi - lo) * u.astype(np.float64))).astype(np.float32)


def waypoints(seed: int, n: int) -> np.ndarray:
    """[n, 4] float32 PID waypoints (x, y, z, yaw): U[-2, 2]^2 x U[0.2, 2] m, yaw 0."""
    idx = np.arange(n, dtype=np.uint64)[:, None]
    u = uniform(seed, S_WAYPOINT, 0, idx, np.arange(3, dtype=np.uint64)[None, :]).astype(np.float64)
    lo = np.array([-2, -2, 0.2])
    hi = np.array([2, 2, 2.0])
    out = np.zeros((n, 4), np.float32)
    out[:, :3] = lo + (hi - lo) * u
    return out


def mixed_actions(swarm: Swarm, seed: int, step: int, hover_rpm: float) -> np.ndarray:
    """Per-drone action for a batch whose envs mix RPM and PID: RPMs where the env takes RPM
    actions, the env's fixed waypoints where it takes PID actions."""
    a = rpm_actions(seed, swarm.n, step, hover_rpm)
    pid = np.repeat(swarm.act_type == ACT_PID, swarm.drones_per_env)
    a[pid] = waypoints(seed, swarm.n)[pid]
    return a


S_ACT_TYPE, S_ACT_EXT, S_DR = 10, 11, 12
DR_PARAMS = 40


def dr_table(seed: int, n_envs: int, dt_ctrl: float = 1.0 / 48.0, depth: int = 3,
             wind_bits: int = 15) -> np.ndarray:
    """float32 [n_envs, 32] domain-randomization rows drawn from the recommended ranges of
    the paper's table for CF2X (factors U(1 - a, 1 + a)): mass and inertia x[0.8, 1.2], arm
    x[0.98, 1.02], k_f and k_m x[0.85, 1.15], drag, C_gnd and C1 x[0.7, 1.3], per-motor bias
    x[0.95, 1.05], MAX_RPM x[0.95, 1.05], g x[0.98, 1.02], motor lag U[5, 50] ms, action
    latency U[0, 50] ms as whole control steps (below `depth`); wind (the model bits given)
    with a horizontal steady wind of magnitude U(0, 1) m/s, 1/2 rho C_d A U[5e-4, 2e-3] kg/m,
    gusts p U[0.02, 0.1] per step, A U[0.02, 0.08] N, duration U[0.1, 0.5] s, Dryden sigma
    U[0.1, 0.5] m/s, V U[1, 5] m/s, h U[0.5, 2] m, sinusoid A U[0.005, 0.02] N,
    w U[1, 6] rad/s; sensors: noise sigmas 1 cm, 5 cm/s, 1 degree, 0.05 rad/s, sensor latency
    U[0, 20] ms as whole control steps (0 or 1). The layout is that of MDG_DR_PARAMS in
    include/mdg.h."""
    e = np.arange(n_envs, dtype=np.uint64)[:, None]
    u = uniform(seed, S_DR, 0, e, np.arange(DR_PARAMS, dtype=np.uint64)[None, :]).astype(np.float64)
    r = np.zeros((n_envs, DR_PARAMS))

    def U(col, lo, hi):
        return lo + (hi - lo) * u[:, col]
    r[:, 0] = U(0, 0.8, 1.2)
    for k in range(3):
        r[:, 1 + k] = U(1 + k, 0.8, 1.2)
    r[:, 4] = U(4, 0.98, 1.02)
    r[:, 5], r[:, 6] = U(5, 0.85, 1.15), U(6, 0.85, 1.15)
    for k in (7, 8, 9, 10):
        r[:, k] = U(k, 0.7, 1.3)
    r[:, 11] = U(11, 0.95, 1.05)
    for k in range(4):
        r[:, 12 + k] = U(12 + k, 0.95, 1.05)
    r[:, 16] = U(16, 0.98, 1.02)
    r[:, 17] = U(17, 0.005, 0.05)
    r[:, 18] = np.minimum(np.floor(U(18, 0.0, 0.05) / dt_ctrl + 0.5), depth - 1)
    r[:, 19] = wind_bits
    speed, heading = U(19, 0.0, 1.0), U(20, 0.0, 2 * np.pi)
    r[:, 20], r[:, 21] = speed * np.cos(heading), speed * np.sin(heading)
    r[:, 23] = U(21, 5e-4, 2e-3)
    r[:, 24], r[:, 25], r[:, 26] = U(22, 0.02, 0.1), U(23, 0.02, 0.08), U(24, 0.1, 0.5)
    r[:, 27], r[:, 28], r[:, 31] = U(25, 0.1, 0.5), U(26, 1.0, 5.0), U(27, 0.5, 2.0)
    r[:, 29], r[:, 30] = U(28, 0.005, 0.02), U(29, 1.0, 6.0)
    r[:, 32], r[:, 33], r[:, 34], r[:, 35] = 0.01, 0.05, np.radians(1.0), 0.05
    r[:, 36] = np.minimum(np.floor(U(30, 0.0, 0.02) / dt_ctrl + 0.5), 1.0)
    return r.astype(np.float32)


def all_action_types(seed: int, n_envs: int) -> np.ndarray:
    """uint8 [n_envs]: each environment's action type drawn uniformly from the six types."""
    u = uniform(seed, S_ACT_TYPE, 0, np.arange(n_envs, dtype=np.uint64), 0).astype(np.float64)
    pick = np.minimum((u * len(ALL_ACTION_TYPES)).astype(np.int64), len(ALL_ACTION_TYPES) - 1)
    return np.asarray(ALL_ACTION_TYPES, np.uint8)[pick]


def typed_actions(drones_per_env: np.ndarray, act_types: np.ndarray, seed: int, step: int, hover_rpm: float,
                  hover_thrust: float) -> np.ndarray:
    """[n, 4] float32 actions for per-environment action types (hover_rpm and hover_thrust
    are the caller's scales):
    RPM        U[0.9, 1.1] x hover_rpm per motor
    PID        waypoints (see waypoints)
    RPM_NORM   U[-1.2, 1.2] per motor (beyond [-1, 1] to exercise the clip)
    ONE_D_RPM  U[-1.2, 1.2] in the first value, the others U[-1.2, 1.2] too (ignored)
    VEL        U[-1, 1]^3 m/s body velocity, U[-1, 1] rad/s yaw rate
    ATTITUDE   U[0.8, 1.2] x hover_thrust, roll and pitch U[-0.3, 0.3] rad, yaw rate U[-1, 1]."""
    n = int(np.sum(drones_per_env))
    per = np.repeat(np.asarray(act_types), drones_per_env)
    idx = np.arange(n, dtype=np.uint64)[:, None]
    comp = np.arange(4, dtype=np.uint64)[None, :]
    u = uniform(seed, S_ACT_EXT, step, idx, comp).astype(np.float64)
    out = np.zeros((n, 4), np.float64)
    rpm = rpm_actions(seed, n, step, hover_rpm).astype(np.float64)
    wp = waypoints(seed, n).astype(np.float64)
    out[per == ACT_RPM] = rpm[per == ACT_RPM]
    out[per == ACT_PID] = wp[per == ACT_PID]
    norm = -1.2 + 2.4 * u
    for t in (ACT_RPM_NORM, ACT_ONE_D_RPM):
        out[per == t] = norm[per == t]
    vel = np.concatenate([-1.0 + 2.0 * u[:, 0:3], -1.0 + 2.0 * u[:, 3:4]], axis=1)
    out[per == ACT_VEL] = vel[per == ACT_VEL]
    att = np.stack([hover_thrust * (0.8 + 0.4 * u[:, 0]), -0.3 + 0.6 * u[:, 1], -0.3 + 0.6 * u[:, 2],
                    -1.0 + 2.0 * u[:, 3]], axis=1)
    out[per == ACT_ATTITUDE] = att[per == ACT_ATTITUDE]
    return out.astype(np.float32)


S_MLP = 9


def mlp_init(seed: int, dims=(64, 256, 256, 256, 32)):
    """Initial surrogate weights: W_l ~ U[-b, b] with b = sqrt(6 / fan_in) (He uniform), b_l = 0;
    float32 arrays [(W [out, in], b [out]), ...], drawn counter-based per (layer, row, col)."""
    out = []
    for l, (fi, fo) in enumerate(zip(dims[:-1], dims[1:])):
        bound = math.sqrt(6.0 / fi)
        u = uniform(seed, S_MLP, l, np.arange(fo, dtype=np.uint64)[:, None], np.arange(fi, dtype=np.uint64)[None, :])
        out.append(((bound * (2.0 * u.astype(np.float64) - 1.0)).astype(np.float32), np.zeros(fo, np.float32)))
    return out


def random_states(seed: int, n: int, pos_scale=1.0, vel_scale=1.0, rate_scale=3.0, z0=1.0):
    """Generic tumbling states for parity tests: p around (0, 0, z0), any attitude, nonzero
    velocity and body rate. Returns (p, q, v, w) float32."""
    idx = np.arange(n, dtype=np.uint64)[:, None]
    c3 = np.arange(3, dtype=np.uint64)[None, :]
    p = uniform_range(-pos_scale, pos_scale, seed, S_POS, 1, idx, c3).astype(np.float64)
    p[:, 2] += z0
    rpy = uniform_range(-math.pi, math.pi, seed, S_ATT, 1, idx, c3).astype(np.float64)
    rpy[:, 1] *= 0.45
    v = uniform_range(-vel_scale, vel_scale, seed, S_VEL, 1, idx, c3)
    w = uniform_range(-rate_scale, rate_scale, seed, S_VEL, 2, idx, c3)
    return p.astype(np.float32), quat_from_rpy(rpy.astype(np.float32)), v, w
