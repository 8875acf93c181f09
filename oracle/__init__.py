"""FP64 CPU oracle of the batched Crazyflie 2.x dynamics step (test infrastructure).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The CUDA
library and its Python binding never import, link or call it, and the two share
no code: the oracle keeps its own constant table, its own formulas and its own
build.

The arithmetic lives in ``mdg_oracle.c`` (plain double-precision loops written
from the paper's Section 3.1 equations, the exponential map of Section 3.2 and
the PID of Section 4.2); this module compiles it with gcc and exposes it to
numpy. ``mlp.py`` holds the FP64 reference of the learned surrogate.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

GND, DRAG, DW = 1, 2, 4
ACT_RPM, ACT_PID = 0, 1
ACT_RPM_NORM, ACT_ONE_D_RPM, ACT_VEL, ACT_ATTITUDE = 3, 4, 5, 6
FRAME_X, FRAME_P = 0, 1
EULER, RK4 = 0, 1
GND_COM, GND_ROTOR = 0, 1
CTRL_PID, CTRL_DSL = 0, 1
DR_PARAMS, WIND_STATE = 40, 8
(DR_MASS, DR_J, DR_ARM, DR_KF, DR_KM, DR_CXY, DR_CZ, DR_CGND, DR_C1, DR_MAXRPM, DR_BIAS, DR_G, DR_TAU, DR_DELAY,
 DR_WIND, DR_VWIND, DR_KDRAG, DR_GUST_P, DR_GUST_A, DR_GUST_T, DR_DRY_SIGMA, DR_DRY_V, DR_SIN_A, DR_SIN_W,
 DR_DRY_H) = (0, 1, 4, 5, 6, 7, 8, 9, 10, 11, 12, 16, 17, 18, 19, 20, 23, 24, 25, 26, 27, 28, 29, 30, 31)
DR_NOISE_P, DR_NOISE_V, DR_NOISE_RPY, DR_NOISE_W, DR_OBS_DELAY = 32, 33, 34, 35, 36
WIND_CONSTANT, WIND_GUST, WIND_DRYDEN, WIND_SINUSOIDAL = 1, 2, 4, 8
STREAM_WIND, STREAM_OBS = 21, 22


class _DR(ctypes.Structure):
    _fields_ = [("env_dr", ctypes.POINTER(ctypes.c_double)), ("motor", ctypes.POINTER(ctypes.c_double)),
                ("hist", ctypes.POINTER(ctypes.c_double)), ("depth", ctypes.c_int32),
                ("wind", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.c_uint64),
                ("obs_bias", ctypes.POINTER(ctypes.c_double))]


class Randomization:
    """Domain-randomization and wind inputs and state of orc_control_steps: env_dr
    [n_envs, DR_PARAMS] (neutral: factors 1, no lag, no delay, no wind), motor [n, 4] and
    hist [depth, n, 4] (NaN: not set), wind [n_envs, WIND_STATE] (Dryden 0, gust idle,
    step 0); all float64, updated in place by control_steps. obs_bias: None or [n, 12], the
    sticky per-episode observation bias added to the KIN channels (orc_obs_bias)."""

    def __init__(self, n_envs: int, n: int, depth: int = 1, seed: int = 0):
        self.env_dr = neutral_dr(n_envs)
        self.motor = np.full((n, 4), np.nan)
        self.hist = np.full((depth, n, 4), np.nan)
        self.wind = np.zeros((n_envs, WIND_STATE))
        self.wind[:, 3] = -1.0
        self.seed = int(seed)
        self.obs_bias = None

    def struct(self) -> _DR:
        for a in (self.env_dr, self.motor, self.hist, self.wind):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        if self.obs_bias is not None:
            assert self.obs_bias.dtype == np.float64 and self.obs_bias.flags.c_contiguous
            assert self.obs_bias.shape == (self.motor.shape[0], 12)
        return _DR(_dptr(self.env_dr), _dptr(self.motor), _dptr(self.hist), self.hist.shape[0], _dptr(self.wind),
                   ctypes.c_uint64(self.seed), _dptr(self.obs_bias) if self.obs_bias is not None else None)


def neutral_dr(n_envs: int) -> np.ndarray:
    """[n_envs, DR_PARAMS] rows that change nothing: every factor 1, no lag, no delay, no wind."""
    r = np.zeros((n_envs, DR_PARAMS))
    r[:, [DR_MASS, DR_J, DR_J + 1, DR_J + 2, DR_ARM, DR_KF, DR_KM, DR_CXY, DR_CZ, DR_CGND, DR_C1, DR_MAXRPM,
          DR_BIAS, DR_BIAS + 1, DR_BIAS + 2, DR_BIAS + 3, DR_G]] = 1.0
    r[:, DR_GUST_T] = 1.0
    r[:, DR_DRY_H] = 1.0
    return r

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile mdg_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of the oracle's own ``orc_params`` struct (field order as in mdg_oracle.c)."""
    _fields_ = [(n, ctypes.c_double) for n in (
        "mass", "arm", "thrust2weight", "Jxx", "Jyy", "Jzz", "kf", "km", "prop_radius", "g",
        "c_gnd", "h_clip", "c_xy", "c_z", "dw_c1", "dw_c2", "dw_c3", "dw_max_xy", "dw_dz_min")] + [
        ("pos_kp", ctypes.c_double * 3), ("pos_ki", ctypes.c_double * 3), ("pos_kd", ctypes.c_double * 3),
        ("pos_iclamp", ctypes.c_double),
        ("att_kp", ctypes.c_double * 3), ("att_ki", ctypes.c_double * 3), ("att_kd", ctypes.c_double * 3),
        ("att_iclamp", ctypes.c_double),
        ("dt_sim", ctypes.c_double), ("dt_ctrl", ctypes.c_double),
        ("sp_rate_pos", ctypes.c_double), ("sp_rate_yaw", ctypes.c_double),
        ("frame", ctypes.c_int32), ("integrator", ctypes.c_int32), ("gnd_heights", ctypes.c_int32),
        ("controller", ctypes.c_int32)]

    def to_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else float(v)
        return out


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            sig = {
                "orc_params_size": ([], ctypes.c_int),
                "orc_params_cf2x": ([P], None),
                "orc_params_cf2p": ([P], None),
                "orc_params_race": ([P], None),
                "orc_env_deriv": ([P, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D], None),
                "orc_substep_rk4": ([P, ctypes.c_int, _D, _D, ctypes.c_int, _D, ctypes.c_double, _D], None),
                "orc_hover_rpm": ([P], ctypes.c_double),
                "orc_max_rpm": ([P], ctypes.c_double),
                "orc_quat_mul": ([_D, _D, _D], None),
                "orc_rotation": ([_D, _D], None),
                "orc_rpy": ([_D, _D], None),
                "orc_motor": ([P, _D, _D, _D], None),
                "orc_rotor_position": ([P, ctypes.c_int, _D], None),
                "orc_env_forces": ([P, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D], None),
                "orc_substep": ([P, ctypes.c_int, _D, _D, ctypes.c_int, _D, ctypes.c_double, _D], None),
                "orc_allocation_matrix": ([P, _D], None),
                "orc_pid": ([P, _D, _D, _D, _D, _D, _D], None),
                "orc_pid_ff": ([P, _D, _D, _D, _D, _D, _D, _D, _D], None),
                "orc_dsl_setpoint": ([P, _D, _D, _D], None),
                "orc_controller_dsl": ([P], None),
                "orc_normalized_rpm": ([P, ctypes.c_double], ctypes.c_double),
                "orc_action_to_rpm": ([P, ctypes.c_int, _D, _D, _D, _D, _D], None),
                "orc_kin": ([_D, _D, _D], None),
                "orc_knn": ([ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, _I, _D], None),
                "orc_control_steps": ([P, ctypes.c_int, _I, _I, _I, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                       _D, _I, _D, _D, ctypes.POINTER(_DR)], ctypes.c_int),
                "orc_uniform": ([ctypes.c_uint64] * 5, ctypes.c_double),
                "orc_splitmix64": ([ctypes.c_uint64], ctypes.c_uint64),
                "orc_reset_state": ([_D, _D, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _D], None),
                "orc_obs_bias": ([_D, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _D], None),
                "orc_params_randomized": ([P, _D, P], None),
                "orc_wind_step": ([P, _D, _D, ctypes.c_uint64, ctypes.c_int64, _D, _D], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            if L.orc_params_size() != ctypes.sizeof(Params):
                raise RuntimeError("oracle Params struct does not match orc_params")
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cf2x() -> Params:
    """Default CF2X parameters of the oracle (its own table)."""
    p = Params()
    lib().orc_params_cf2x(ctypes.byref(p))
    return p


def cf2p() -> Params:
    """CF2P: the CF2X parameters with the + rotor layout."""
    p = Params()
    lib().orc_params_cf2p(ctypes.byref(p))
    return p


def race() -> Params:
    """RACE parameters of the oracle (its own table; readings in mdg_oracle.c)."""
    p = Params()
    lib().orc_params_race(ctypes.byref(p))
    return p


def hover_rpm(p: Params) -> float:
    return lib().orc_hover_rpm(ctypes.byref(p))


def max_rpm(p: Params) -> float:
    return lib().orc_max_rpm(ctypes.byref(p))


def quat_mul(a, b) -> np.ndarray:
    a, b = _f64(a), _f64(b)
    out = np.zeros(4)
    lib().orc_quat_mul(_dptr(a), _dptr(b), _dptr(out))
    return out


def rotation(q) -> np.ndarray:
    q = _f64(q)
    R = np.zeros(9)
    lib().orc_rotation(_dptr(q), _dptr(R))
    return R.reshape(3, 3)


def rpy(q) -> np.ndarray:
    q = _f64(q)
    out = np.zeros(3)
    lib().orc_rpy(_dptr(q), _dptr(out))
    return out


def motor(p: Params, rpm):
    rpm = _f64(rpm)
    T = ctypes.c_double()
    tau = np.zeros(3)
    lib().orc_motor(ctypes.byref(p), _dptr(rpm), ctypes.byref(T), _dptr(tau))
    return T.value, tau


def rotor_position(p: Params, i: int) -> np.ndarray:
    """Body-frame position of rotor i (read from the torque equations of Section 3.1.2)."""
    r = np.zeros(3)
    lib().orc_rotor_position(ctypes.byref(p), int(i), _dptr(r))
    return r


def _ext(f_ext, n):
    if f_ext is None:
        return None
    f = _f64(f_ext)
    assert f.shape == (n, 3)
    return f


def env_forces(p: Params, x, rpm, flags: int, f_ext=None):
    """World force (gravity included) [N,3] and body torque [N,3] for one env (plus an
    external world-frame force f_ext [N,3])."""
    x, rpm = _f64(x), _f64(rpm)
    N = x.shape[0]
    F = np.zeros((N, 3))
    tau = np.zeros((N, 3))
    fe = _ext(f_ext, N)
    lib().orc_env_forces(ctypes.byref(p), N, _dptr(x), _dptr(rpm), int(flags),
                         _dptr(fe) if fe is not None else None, _dptr(F), _dptr(tau))
    return F, tau


def substep(p: Params, x, rpm, flags: int, dt: float | None = None, f_ext=None) -> np.ndarray:
    """One substep of one environment: x [N,13], rpm [N,4] -> x' [N,13]."""
    x, rpm = _f64(x), _f64(rpm)
    out = np.zeros_like(x)
    fe = _ext(f_ext, x.shape[0])
    lib().orc_substep(ctypes.byref(p), x.shape[0], _dptr(x), _dptr(rpm), int(flags),
                      _dptr(fe) if fe is not None else None, p.dt_sim if dt is None else float(dt), _dptr(out))
    return out


def env_deriv(p: Params, x, rpm, flags: int, f_ext=None) -> np.ndarray:
    """Time derivative of one environment's state: x [N,13], rpm [N,4] -> dx/dt [N,13]."""
    x, rpm = _f64(x), _f64(rpm)
    out = np.zeros_like(x)
    fe = _ext(f_ext, x.shape[0])
    lib().orc_env_deriv(ctypes.byref(p), x.shape[0], _dptr(x), _dptr(rpm), int(flags),
                        _dptr(fe) if fe is not None else None, _dptr(out))
    return out


def substep_rk4(p: Params, x, rpm, flags: int, dt: float | None = None, f_ext=None) -> np.ndarray:
    """One classical RK4 substep of one environment: x [N,13], rpm [N,4] -> x' [N,13]."""
    x, rpm = _f64(x), _f64(rpm)
    out = np.zeros_like(x)
    fe = _ext(f_ext, x.shape[0])
    lib().orc_substep_rk4(ctypes.byref(p), x.shape[0], _dptr(x), _dptr(rpm), int(flags),
                          _dptr(fe) if fe is not None else None, p.dt_sim if dt is None else float(dt), _dptr(out))
    return out


def allocation_matrix(p: Params) -> np.ndarray:
    M = np.zeros(16)
    lib().orc_allocation_matrix(ctypes.byref(p), _dptr(M))
    return M.reshape(4, 4)


def pid(p: Params, x, integ, wp):
    """One PID call: returns (rpm[4], pos_err[3], yaw_err, new integ[6])."""
    x, wp = _f64(x), _f64(wp)
    integ = _f64(integ).copy()
    rpm = np.zeros(4)
    pe = np.zeros(3)
    ye = ctypes.c_double()
    lib().orc_pid(ctypes.byref(p), _dptr(x), _dptr(integ), _dptr(wp), _dptr(rpm), _dptr(pe), ctypes.byref(ye))
    return rpm, pe, ye.value, integ


def controller_dsl(p: Params) -> Params:
    """The DSL controller's gains, clamps and rate limits applied to a copy of p."""
    q = Params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(Params))
    lib().orc_controller_dsl(ctypes.byref(q))
    return q


def new_setpoints(n: int) -> np.ndarray:
    """[n, 4] DSL setpoints not yet set (NaN): each starts at its drone's position and yaw."""
    return np.full((n, 4), np.nan)


def dsl_setpoint(p: Params, x, wp, sp):
    """One step of the setpoint limiter; returns the new setpoint [4]."""
    x, wp = _f64(x), _f64(wp)
    sp = _f64(sp).copy()
    lib().orc_dsl_setpoint(ctypes.byref(p), _dptr(x), _dptr(wp), _dptr(sp))
    return sp


def pid_ff(p: Params, x, integ, wp, a_ff=None, sp=None):
    """One controller call with an optional feed-forward acceleration and DSL setpoint:
    returns (rpm[4], pos_err[3], yaw_err, new integ[6], new setpoint[4] or None)."""
    x, wp = _f64(x), _f64(wp)
    integ = _f64(integ).copy()
    sp = None if sp is None else _f64(sp).copy()
    ff = None if a_ff is None else _f64(a_ff)
    rpm, pe, ye = np.zeros(4), np.zeros(3), ctypes.c_double()
    lib().orc_pid_ff(ctypes.byref(p), _dptr(x), _dptr(integ), _dptr(sp) if sp is not None else None, _dptr(wp),
                     _dptr(ff) if ff is not None else None, _dptr(rpm), _dptr(pe), ctypes.byref(ye))
    return rpm, pe, ye.value, integ, sp


def normalized_rpm(p: Params, a: float) -> float:
    return lib().orc_normalized_rpm(ctypes.byref(p), float(a))


def action_to_rpm(p: Params, act_type: int, x, integ, act):
    """One drone's action -> (rpm [4], updated integ [6]) for any action type (no DSL setpoint)."""
    x, act = _f64(x), _f64(act)
    integ = _f64(integ).copy()
    rpm = np.zeros(4)
    lib().orc_action_to_rpm(ctypes.byref(p), int(act_type), _dptr(x), _dptr(integ), None, _dptr(act), _dptr(rpm))
    return rpm, integ


def kin(x, a_prev) -> np.ndarray:
    x, a_prev = _f64(x), _f64(a_prev)
    out = np.zeros(20)
    lib().orc_kin(_dptr(x), _dptr(a_prev), _dptr(out))
    return out


def knn(x_env, j: int, idx_base: int = 0):
    """4-NN of drone j inside one environment x_env [N,13]: (idx[4] int32, rel[24])."""
    x_env = _f64(x_env)
    idx = np.zeros(4, dtype=np.int32)
    rel = np.zeros(24)
    lib().orc_knn(x_env.shape[0], _dptr(x_env), int(j), int(idx_base), _iptr(idx), _dptr(rel))
    return idx, rel


def splitmix64(z: int) -> int:
    """The oracle's SplitMix64 round: the generator's output for the state z before its
    increment by the golden gamma (so z = k * gamma gives the (k+1)-th output from state 0)."""
    return int(lib().orc_splitmix64(ctypes.c_uint64(z % (1 << 64))))


def reset_state(nominal, ranges, seed: int, episode: int, drone: int) -> np.ndarray:
    """Initial state [13] of one drone for one episode (orc_reset_state): nominal [x, y, z,
    yaw], ranges [p0 (m), rpy0 (rad), v0 (m/s)] half-widths of the uniform perturbations."""
    nom, rng = _f64(nominal), _f64(ranges)
    x = np.zeros(13)
    lib().orc_reset_state(_dptr(nom), _dptr(rng), seed, episode, drone, _dptr(x))
    return x


def obs_bias(sigmas, seed: int, episode: int, drone: int) -> np.ndarray:
    """Sticky per-episode observation bias [12] of one drone (orc_obs_bias): sigmas [position,
    roll/pitch/yaw, velocity, body rate]."""
    sg = _f64(sigmas)
    b = np.zeros(12)
    lib().orc_obs_bias(_dptr(sg), seed, episode, drone, _dptr(b))
    return b


def uniform(seed: int, stream: int, step: int, index: int, comp: int) -> float:
    """The oracle's counter-based U[0, 1) (SplitMix64 rounds over the five counters)."""
    return lib().orc_uniform(seed, stream, step, index, comp)


def params_randomized(p: Params, row) -> Params:
    q = Params()
    r = _f64(row)
    lib().orc_params_randomized(ctypes.byref(p), _dptr(r), ctypes.byref(q))
    return q


def wind_step(p: Params, row, ws, seed: int, env: int):
    """One control step of an environment's wind: returns (F_dir [3], v_wind [3]); ws
    (float64 [WIND_STATE]) is updated in place."""
    r = _f64(row)
    assert ws.dtype == np.float64 and ws.flags.c_contiguous
    F, v = np.zeros(3), np.zeros(3)
    lib().orc_wind_step(ctypes.byref(p), _dptr(r), _dptr(ws), seed, env, _dptr(F), _dptr(v))
    return F, v


def control_steps(p: Params, env_off, env_flags, env_act, x, integ, a_prev, actions, n_sub: int,
                  obs: bool = False, setpoint=None, dr: "Randomization | None" = None):
    """K control steps over a CSR batch. x [n,13], integ [n,6], a_prev [n,4] and actions [K,n,4]
    (float64). Returns (x, integ, a_prev) updated copies, plus (kin, nbr_idx, nbr_rel) when obs.
    setpoint: float64 C-contiguous [n,4] DSL setpoints, updated in place (required with the
    DSL controller)."""
    if setpoint is not None:
        assert isinstance(setpoint, np.ndarray) and setpoint.dtype == np.float64 and setpoint.flags.c_contiguous
    env_off = np.ascontiguousarray(env_off, dtype=np.int32)
    env_flags = np.ascontiguousarray(env_flags, dtype=np.int32)
    env_act = np.ascontiguousarray(env_act, dtype=np.int32)
    x = _f64(x).copy()
    integ = _f64(integ).copy()
    a_prev = _f64(a_prev).copy()
    actions = _f64(actions)
    n = x.shape[0]
    K = actions.shape[0]
    assert actions.shape == (K, n, 4) and integ.shape == (n, 6) and a_prev.shape == (n, 4)
    n_envs = env_off.shape[0] - 1
    kin_o = nbr_i = nbr_r = None
    if obs:
        kin_o = np.zeros((n, 20))
        nbr_i = np.zeros((n, 4), dtype=np.int32)
        nbr_r = np.zeros((n, 24))
    rc = lib().orc_control_steps(ctypes.byref(p), n_envs, _iptr(env_off), _iptr(env_flags), _iptr(env_act),
                                 _dptr(x), _dptr(integ), _dptr(a_prev), _dptr(actions), K, int(n_sub),
                                 _dptr(kin_o) if obs else None, _iptr(nbr_i) if obs else None,
                                 _dptr(nbr_r) if obs else None, _dptr(setpoint) if setpoint is not None else None,
                                 ctypes.byref(dr.struct()) if dr is not None else None)
    if rc != 0:
        raise ValueError("orc_control_steps rejected its arguments")
    if obs:
        return x, integ, a_prev, kin_o, nbr_i, nbr_r
    return x, integ, a_prev


def control_steps_into(p: Params, env_off, env_flags, env_act, x, integ, a_prev, actions, n_sub: int,
                       kin, nbr_idx, nbr_rel, setpoint=None, dr: "Randomization | None" = None) -> None:
    """control_steps with observations on caller-owned C-contiguous arrays: x [n,13], integ
    [n,6], a_prev [n,4] (float64) are updated in place, kin [n,20], nbr_rel [n,24] (float64)
    and nbr_idx [n,4] (int32) written; env_off, env_flags, env_act int32. The same C routine
    without the wrapper's copies (for timing the oracle on many threads)."""
    for a, dt in ((x, np.float64), (integ, np.float64), (a_prev, np.float64), (actions, np.float64),
                  (kin, np.float64), (nbr_rel, np.float64), (nbr_idx, np.int32), (env_off, np.int32),
                  (env_flags, np.int32), (env_act, np.int32)):
        assert a.dtype == dt and a.flags.c_contiguous
    n = x.shape[0]
    K = actions.shape[0]
    assert actions.shape == (K, n, 4) and kin.shape == (n, 20) and nbr_idx.shape == (n, 4)
    rc = lib().orc_control_steps(ctypes.byref(p), env_off.shape[0] - 1, _iptr(env_off), _iptr(env_flags),
                                 _iptr(env_act), _dptr(x), _dptr(integ), _dptr(a_prev), _dptr(actions), K, int(n_sub),
                                 _dptr(kin), _iptr(nbr_idx), _dptr(nbr_rel),
                                 _dptr(setpoint) if setpoint is not None else None,
                                 ctypes.byref(dr.struct()) if dr is not None else None)
    if rc != 0:
        raise ValueError("orc_control_steps rejected its arguments")
