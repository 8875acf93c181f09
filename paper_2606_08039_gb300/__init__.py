"""GB300-native batched multi-drone dynamics (MuJoCo-Drones-Gym hot path, arxiv 2606.08039).

Thin Python binding of the C ABI in include/mdg.h. It only marshals arguments: torch
tensors provide device memory and streams, every computation runs in the CUDA kernels
of libmdg.so. There is no CPU fallback: if the library is not built the first call
raises.

    import paper_2606_08039_gb300 as mdg
    h = mdg.Handle(drones_per_env, model_flags)          # one handle per batch layout
    state = mdg.pack_state(p, q, v, w, device="cuda")    # [6, n, 4] float32 planes
    h.step(state, action, mdg.ACT_PID, n_substeps=5)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads  # noqa: F401  (seeded synthetic inputs)

GND, DRAG, DW = 1, 2, 4
ACT_RPM, ACT_PID, ACT_MIXED = 0, 1, 2
ACT_RPM_NORM, ACT_ONE_D_RPM, ACT_VEL, ACT_ATTITUDE = 3, 4, 5, 6
STATUS_NONFINITE = 1
STATUS_TIMEOUT = 2
SCHED_DYNAMIC, SCHED_STATIC = 0, 1
STATUS_BOUNDS = 4
MLP_PATH_MMA_SYNC, MLP_PATH_TCGEN05, MLP_PATH_TCGEN05_PAIRS = 0, 1, 2
STATE_PLANES = 6
KIN_DIM = 20
NBR_K = 4
NBR_FEAT = 6
MAX_ENV_DRONES = 1024

OK, ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_UNSUPPORTED, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
FRAME_X, FRAME_P = 0, 1
INTEGRATOR_EULER, INTEGRATOR_RK4 = 0, 1
GND_COM, GND_ROTOR = 0, 1
CTRL_PID, CTRL_DSL = 0, 1
CAM_H, CAM_W = 48, 64
DR_PARAMS, WIND_STATE, MAX_HIST_DEPTH = 40, 8, 16
(DR_MASS, DR_J, DR_ARM, DR_KF, DR_KM, DR_CXY, DR_CZ, DR_CGND, DR_C1, DR_MAXRPM, DR_BIAS, DR_G, DR_TAU, DR_DELAY,
 DR_WIND, DR_VWIND, DR_KDRAG, DR_GUST_P, DR_GUST_A, DR_GUST_T, DR_DRY_SIGMA, DR_DRY_V, DR_SIN_A, DR_SIN_W,
 DR_DRY_H) = (0, 1, 4, 5, 6, 7, 8, 9, 10, 11, 12, 16, 17, 18, 19, 20, 23, 24, 25, 26, 27, 28, 29, 30, 31)
DR_NOISE_P, DR_NOISE_V, DR_NOISE_RPY, DR_NOISE_W, DR_OBS_DELAY = 32, 33, 34, 35, 36
WIND_CONSTANT, WIND_GUST, WIND_DRYDEN, WIND_SINUSOIDAL, WIND_COMBINED = 1, 2, 4, 8, 15
OBS_NONE, OBS_LAST, OBS_EVERY_STEP = 0, 1, 2
MLP_IN, MLP_IN_PAD, MLP_HIDDEN, MLP_OUT, MLP_OUT_PAD = 41, 64, 256, 13, 32
MLP_DIMS = (MLP_IN_PAD, MLP_HIDDEN, MLP_HIDDEN, MLP_HIDDEN, MLP_OUT_PAD)
MLP_PARAMS = 156448

_HERE = os.path.dirname(os.path.abspath(__file__))
# MDG_DEBUG_LIBRARY=1 loads the index-checking debug build (build_library(debug=True))
LIB_PATH = os.path.join(_HERE, "_lib", "libmdg_debug.so" if os.environ.get("MDG_DEBUG_LIBRARY") == "1" else "libmdg.so")

# Every symbol include/mdg.h declares, with its ctypes signature.
_VP = ctypes.c_void_p
_SIGNATURES = {
    "mdg_constants_cf2x": ([_VP], ctypes.c_int),
    "mdg_constants_cf2p": ([_VP], ctypes.c_int),
    "mdg_constants_race": ([_VP], ctypes.c_int),
    "mdg_controller_dsl": ([_VP], ctypes.c_int),
    "mdg_set_setpoints": ([_VP, _VP], ctypes.c_int),
    "mdg_render": ([_VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_set_randomization": ([_VP, _VP, _VP, _VP, ctypes.c_int32, _VP, ctypes.c_uint64], ctypes.c_int),
    "mdg_pid_ff": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_constants_size": ([], ctypes.c_int),
    "mdg_hover_rpm": ([_VP], ctypes.c_double),
    "mdg_max_rpm": ([_VP], ctypes.c_double),
    "mdg_create": ([ctypes.c_int32, _VP, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "mdg_destroy": ([_VP], ctypes.c_int),
    "mdg_num_drones": ([_VP], ctypes.c_int64),
    "mdg_set_action_types": ([_VP, _VP], ctypes.c_int),
    "mdg_set_block_size": ([_VP, ctypes.c_int32], ctypes.c_int),
    "mdg_get_block_size": ([_VP], ctypes.c_int32),
    "mdg_step": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP], ctypes.c_int),
    "mdg_step_obs": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_pid": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_obs": ([_VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_status": ([_VP, _VP, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "mdg_last_error": ([], ctypes.c_char_p),
    "mdg_rollout": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                     _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_rollout_graph_create": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, _VP, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "mdg_graph_launch": ([_VP, _VP], ctypes.c_int),
    "mdg_graph_destroy": ([_VP], ctypes.c_int),
    "mdg_autotune": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP,
                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "mdg_mlp_create": ([ctypes.c_int32, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "mdg_mlp_destroy": ([_VP], ctypes.c_int),
    "mdg_mlp_get_params": ([_VP, _VP], ctypes.c_int),
    "mdg_mlp_set_params": ([_VP, _VP], ctypes.c_int),
    "mdg_mlp_get_grads": ([_VP, _VP], ctypes.c_int),
    "mdg_mlp_set_normalization": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_mlp_standardize": ([_VP, _VP, _VP, ctypes.c_int64, _VP], ctypes.c_int),
    "mdg_mlp_forward": ([_VP, _VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "mdg_mlp_grad": ([_VP, _VP, _VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "mdg_mlp_adam": ([_VP, ctypes.c_float, _VP], ctypes.c_int),
    "mdg_mlp_set_path": ([_VP, ctypes.c_int32], ctypes.c_int),
    "mdg_mlp_set_wait_limits": ([_VP, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "mdg_mlp_set_train_path": ([_VP, ctypes.c_int32], ctypes.c_int),
    "mdg_transition": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "mdg_mlp_fit_normalization": ([_VP, _VP, _VP, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, _VP, _VP, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64), _VP], ctypes.c_int),
    "mdg_mlp_get_normalization": ([_VP] * 7, ctypes.c_int),
    "mdg_reset": ([_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_uint64, ctypes.c_uint64, _VP], ctypes.c_int),
    "mdg_set_obs_bias": ([_VP, _VP], ctypes.c_int),
    "mdg_set_rollout_schedule": ([_VP, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "mdg_get_rollout_schedule": ([_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "mdg_mlp_status": ([_VP, _VP, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "mdg_features": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_surrogate_step": ([_VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _VP, _VP],
                           ctypes.c_int),
    "mdg_sync": ([_VP, ctypes.c_int32], ctypes.c_int),
    "mdg_step_obs_host": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, _VP], ctypes.c_int),
    "mdg_step_obs_noalloc": ([_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP,
                              _VP, _VP, _VP], ctypes.c_int),
}

_lock = threading.Lock()
_lib = None


class MdgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mdg error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded libmdg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run paper_2606_08039_gb300.build.build_library() "
                                   "(needs nvcc). There is no CPU fallback.")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            if L.mdg_constants_size() != ctypes.sizeof(Constants):
                raise RuntimeError("Constants mirror does not match mdg_constants")
            _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise MdgError(rc, lib().mdg_last_error().decode())


class Constants(ctypes.Structure):
    """Mirror of mdg_constants (include/mdg.h)."""
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

    def with_dsl(self) -> "Constants":
        """A copy with the DSL controller's gains, clamps and setpoint limits (mdg_controller_dsl)."""
        c = Constants()
        ctypes.memmove(ctypes.byref(c), ctypes.byref(self), ctypes.sizeof(Constants))
        _check(lib().mdg_controller_dsl(ctypes.byref(c)))
        return c

    @classmethod
    def cf2x(cls) -> "Constants":
        c = cls()
        _check(lib().mdg_constants_cf2x(ctypes.byref(c)))
        return c

    @classmethod
    def cf2p(cls) -> "Constants":
        c = cls()
        _check(lib().mdg_constants_cf2p(ctypes.byref(c)))
        return c

    @classmethod
    def race(cls) -> "Constants":
        c = cls()
        _check(lib().mdg_constants_race(ctypes.byref(c)))
        return c

    def hover_rpm(self) -> float:
        return lib().mdg_hover_rpm(ctypes.byref(self))

    def max_rpm(self) -> float:
        return lib().mdg_max_rpm(ctypes.byref(self))

    def to_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


# ---------------------------------------------------------------- tensor marshalling
def _torch():
    import torch
    return torch


def _ptr(t, name, dtype, shape=None):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t, name, dtype, shape=None):
    """Pointer of a page-locked (pinned) CPU tensor; the library checks that it is mapped."""
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cpu" or not t.is_pinned():
        raise ValueError(f"{name} must be a pinned CPU tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def sync(stream=None, timeout_ms: int = 1000) -> int:
    """Bounded host-side wait on a stream (mdg_sync): OK, or ERR_TIMEOUT if it is still busy."""
    rc = lib().mdg_sync(_stream(stream), int(timeout_ms))
    if rc not in (OK, ERR_TIMEOUT):
        _check(rc)
    return rc


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def pack_state(p, q, v, w, ip=None, ia=None, a_prev=None, device="cuda"):
    """Lay (p[n,3], q[n,4] (w,x,y,z), v[n,3], w[n,3], PID integrals ip[n,3], ia[n,3],
    last RPMs a_prev[n,4]) out as the library's [6, n, 4] float32 state planes."""
    torch = _torch()

    def T(a, cols):
        if a is None:
            return torch.zeros((n, cols), dtype=torch.float32)
        return torch.as_tensor(np.asarray(a, dtype=np.float32)).reshape(n, cols)

    n = int(np.asarray(p).shape[0])
    p, q, v, w = T(p, 3), T(q, 4), T(v, 3), T(w, 3)
    ip, ia, a_prev = T(ip, 3), T(ia, 3), T(a_prev, 4)
    z = torch.zeros((n, 1), dtype=torch.float32)
    planes = torch.stack([
        torch.cat([p, q[:, :1]], 1),
        torch.cat([q[:, 1:], v[:, :1]], 1),
        torch.cat([v[:, 1:], w[:, :2]], 1),
        torch.cat([w[:, 2:], ip], 1),
        torch.cat([ia, z], 1),
        a_prev,
    ])
    return planes.contiguous().to(device)


def unpack_state(state) -> dict:
    """Inverse of pack_state: a dict of numpy float32 arrays p, q, v, w, ip, ia, a_prev."""
    s = state.detach().cpu().numpy()
    return {"p": s[0, :, 0:3].copy(), "q": np.concatenate([s[0, :, 3:4], s[1, :, 0:3]], 1),
            "v": np.concatenate([s[1, :, 3:4], s[2, :, 0:2]], 1),
            "w": np.concatenate([s[2, :, 2:4], s[3, :, 0:1]], 1),
            "ip": s[3, :, 1:4].copy(), "ia": s[4, :, 0:3].copy(), "a_prev": s[5].copy()}


class Graph:
    """A replayable rollout (mdg_graph); keeps its buffers alive."""

    def __init__(self, g, keep):
        self._g = g
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().mdg_graph_launch(self._g, _stream(stream)))

    def close(self):
        if self._g:
            lib().mdg_graph_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Handle:
    """A batch of environments (mdg_create). Owns the device tables; all state, action and
    observation tensors belong to the caller."""

    def __init__(self, drones_per_env, model_flags, constants: Constants | None = None):
        dpe = np.ascontiguousarray(drones_per_env, dtype=np.int32)
        flg = np.ascontiguousarray(model_flags, dtype=np.uint32)
        if dpe.shape != flg.shape or dpe.ndim != 1:
            raise ValueError("drones_per_env and model_flags must be 1-d arrays of equal length")
        self._h = ctypes.c_void_p()
        self.constants = constants if constants is not None else Constants.cf2x()
        _check(lib().mdg_create(int(dpe.shape[0]), dpe.ctypes.data_as(_VP), flg.ctypes.data_as(_VP),
                                ctypes.byref(self.constants), ctypes.byref(self._h)))
        self.n_envs = int(dpe.shape[0])
        self.n = int(lib().mdg_num_drones(self._h))
        self.drones_per_env = dpe

    # -- lifetime
    def close(self):
        if self._h:
            lib().mdg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration
    def set_action_types(self, per_env):
        a = np.ascontiguousarray(per_env, dtype=np.uint8)
        if a.shape != (self.n_envs,):
            raise ValueError("per_env must have one entry per environment")
        _check(lib().mdg_set_action_types(self._h, a.ctypes.data_as(_VP)))

    def set_setpoints(self, setpoints):
        """Attach the DSL controller's setpoints: a caller-owned float32 [n, 4] (x, y, z, yaw)
        device tensor, NaN where not set yet (new_setpoints); None detaches. The tensor must
        stay alive while attached."""
        torch = _torch()
        self._setpoints = setpoints
        _check(lib().mdg_set_setpoints(self._h, _ptr(setpoints, "setpoints", torch.float32, (self.n, 4))))

    def new_setpoints(self, device="cuda"):
        """float32 [n, 4] setpoints, all NaN (each starts at its drone's position and yaw)."""
        torch = _torch()
        return torch.full((self.n, 4), float("nan"), dtype=torch.float32, device=device)

    def new_randomization_state(self, depth: int = 1, device="cuda"):
        """(motor [n, 4], action_hist [depth, n, 4], wind_state [n_envs, WIND_STATE]) float32
        device tensors in their starting state: rotor speeds and history unset (NaN), wind
        at rest with no gust (phase -1)."""
        torch = _torch()
        motor = torch.full((self.n, 4), float("nan"), dtype=torch.float32, device=device)
        hist = torch.full((depth, self.n, 4), float("nan"), dtype=torch.float32, device=device)
        wind = torch.zeros((self.n_envs, WIND_STATE), dtype=torch.float32, device=device)
        wind[:, 3] = -1.0
        return motor, hist, wind

    def set_randomization(self, env_params, motor=None, action_hist=None, wind_state=None, seed: int = 0):
        """Attach domain randomization (mdg_set_randomization): env_params float32
        [n_envs, DR_PARAMS] and the state tensors of new_randomization_state (kept alive
        while attached). env_params None detaches."""
        torch = _torch()
        if env_params is None:
            self._dr_keep = None
            _check(lib().mdg_set_randomization(self._h, None, None, None, 0, None, 0))
            return
        depth = int(action_hist.shape[0])
        self._dr_keep = (env_params, motor, action_hist, wind_state)
        _check(lib().mdg_set_randomization(
            self._h, _ptr(env_params, "env_params", torch.float32, (self.n_envs, DR_PARAMS)),
            _ptr(motor, "motor", torch.float32, (self.n, 4)),
            _ptr(action_hist, "action_hist", torch.float32, (depth, self.n, 4)), depth,
            _ptr(wind_state, "wind_state", torch.float32, (self.n_envs, WIND_STATE)), int(seed)))

    def reset(self, state, nominal, init_range=None, bias_sigma=None, obs_bias=None, seed: int = 0,
              episode: int = 0, stream=None):
        """Episode reset with the init row of the randomization table (mdg_reset): state
        [6, n, 4] overwritten from nominal [n, 4] (x, y, z, yaw) perturbed uniformly by
        init_range (p m, angles rad, v m/s); obs_bias [n, 12] (optional) drawn with
        bias_sigma (p, angles, v, body rate)."""
        torch = _torch()
        rng = None if init_range is None else (ctypes.c_float * 3)(*[float(v) for v in init_range])
        sig = None if bias_sigma is None else (ctypes.c_float * 4)(*[float(v) for v in bias_sigma])
        _check(lib().mdg_reset(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                               _ptr(nominal, "nominal", torch.float32, (self.n, 4)),
                               ctypes.cast(rng, _VP) if rng is not None else None,
                               ctypes.cast(sig, _VP) if sig is not None else None,
                               None if obs_bias is None else _ptr(obs_bias, "obs_bias", torch.float32, (self.n, 12)),
                               int(seed), int(episode), _stream(stream)))

    def set_obs_bias(self, obs_bias):
        """Attach (None: detach) the sticky observation bias [n, 12] (mdg_set_obs_bias)."""
        torch = _torch()
        self._bias_keep = obs_bias
        _check(lib().mdg_set_obs_bias(self._h, None if obs_bias is None else
                                      _ptr(obs_bias, "obs_bias", torch.float32, (self.n, 12))))

    def set_rollout_schedule(self, mode: int, item_drones: int = 0):
        """The persistent rollout's work distribution (mdg_set_rollout_schedule)."""
        _check(lib().mdg_set_rollout_schedule(self._h, int(mode), int(item_drones)))

    @property
    def rollout_schedule(self):
        """(mode, item_drones) of mdg_get_rollout_schedule."""
        mode, cap = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().mdg_get_rollout_schedule(self._h, ctypes.byref(mode), ctypes.byref(cap)))
        return mode.value, cap.value

    def set_block_size(self, threads_per_block: int):
        _check(lib().mdg_set_block_size(self._h, int(threads_per_block)))

    @property
    def block_size(self) -> int:
        return int(lib().mdg_get_block_size(self._h))

    # -- compute
    def step(self, state, action, action_type: int, n_substeps: int = 5, stream=None):
        torch = _torch()
        _check(lib().mdg_step(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                              _ptr(action, "action", torch.float32, (self.n, 4)), int(action_type),
                              int(n_substeps), _stream(stream)))

    def step_obs(self, state, action, action_type: int, n_substeps, kin, nbr_idx, nbr_rel=None, stream=None):
        torch = _torch()
        _check(lib().mdg_step_obs(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                                  _ptr(action, "action", torch.float32, (self.n, 4)), int(action_type),
                                  int(n_substeps), _ptr(kin, "kin", torch.float32, (self.n, KIN_DIM)),
                                  _ptr(nbr_idx, "nbr_idx", torch.int32, (self.n, NBR_K)),
                                  _ptr(nbr_rel, "nbr_rel", torch.float32, (self.n, NBR_K * NBR_FEAT)),
                                  _stream(stream)))

    def step_obs_host(self, state, action_host, action_type: int, n_substeps, kin_host, nbr_idx_host,
                      nbr_rel_host=None, stream=None):
        """step_obs with the actions and observations in pinned host tensors, read and written
        by the step kernel itself (mdg_step_obs_host); the state stays on the device."""
        torch = _torch()
        _check(lib().mdg_step_obs_host(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                                       _host_ptr(action_host, "action_host", torch.float32, (self.n, 4)),
                                       int(action_type), int(n_substeps),
                                       _host_ptr(kin_host, "kin_host", torch.float32, (self.n, KIN_DIM)),
                                       _host_ptr(nbr_idx_host, "nbr_idx_host", torch.int32, (self.n, NBR_K)),
                                       _host_ptr(nbr_rel_host, "nbr_rel_host", torch.float32,
                                                 (self.n, NBR_K * NBR_FEAT)),
                                       _stream(stream)))

    def pid(self, state, waypoints, rpm_out, pos_err=None, yaw_err=None, stream=None, target_acc=None):
        torch = _torch()
        _check(lib().mdg_pid_ff(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                             _ptr(waypoints, "waypoints", torch.float32, (self.n, 4)),
                             _ptr(target_acc, "target_acc", torch.float32, (self.n, 4)),
                             _ptr(rpm_out, "rpm_out", torch.float32, (self.n, 4)),
                             _ptr(pos_err, "pos_err", torch.float32, (self.n, 3)),
                             _ptr(yaw_err, "yaw_err", torch.float32, (self.n,)), _stream(stream)))

    def new_frames(self, device="cuda", rgba=True, depth=True, seg=True):
        """(rgba uint8 [n, CAM_H, CAM_W, 4], depth float32 [n, CAM_H, CAM_W], seg int32
        [n, CAM_H, CAM_W]) device tensors (None where not asked for)."""
        torch = _torch()
        shp = (self.n, CAM_H, CAM_W)
        return (torch.empty(shp + (4,), dtype=torch.uint8, device=device) if rgba else None,
                torch.empty(shp, dtype=torch.float32, device=device) if depth else None,
                torch.empty(shp, dtype=torch.int32, device=device) if seg else None)

    def render(self, state, rgba=None, depth=None, seg=None, stream=None):
        """Camera frames of every drone (mdg_render); each output may be None."""
        torch = _torch()
        shp = (self.n, CAM_H, CAM_W)
        _check(lib().mdg_render(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                                _ptr(rgba, "rgba", torch.uint8, shp + (4,)), _ptr(depth, "depth", torch.float32, shp),
                                _ptr(seg, "seg", torch.int32, shp), _stream(stream)))

    def obs(self, state, kin, nbr_idx, nbr_rel=None, stream=None):
        torch = _torch()
        _check(lib().mdg_obs(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                             _ptr(kin, "kin", torch.float32, (self.n, KIN_DIM)),
                             _ptr(nbr_idx, "nbr_idx", torch.int32, (self.n, NBR_K)),
                             _ptr(nbr_rel, "nbr_rel", torch.float32, (self.n, NBR_K * NBR_FEAT)),
                             _stream(stream)))

    def status(self, stream=None):
        """(return code, status bits, first non-finite drone or -1); clears the word."""
        bits = ctypes.c_uint32()
        first = ctypes.c_int64()
        rc = lib().mdg_status(self._h, _stream(stream), ctypes.byref(bits), ctypes.byref(first))
        if rc not in (OK, ERR_NONFINITE):
            _check(rc)
        return rc, bits.value, first.value

    def rollout(self, state, actions, action_type: int, n_substeps: int, K: int, obs_mode: int = OBS_NONE,
                kin=None, nbr_idx=None, nbr_rel=None, stream=None):
        """K control steps in one persistent launch (mdg_rollout). `actions` is [K, n, 4]
        (one action per step) or [n, 4] (reused every step)."""
        torch = _torch()
        per_step = actions.dim() == 3
        shape = (K, self.n, 4) if per_step else (self.n, 4)
        lead = (K,) if obs_mode == OBS_EVERY_STEP else ()
        _check(lib().mdg_rollout(
            self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
            _ptr(actions, "actions", torch.float32, shape), int(per_step), int(action_type), int(n_substeps), int(K),
            int(obs_mode), _ptr(kin, "kin", torch.float32, lead + (self.n, KIN_DIM)),
            _ptr(nbr_idx, "nbr_idx", torch.int32, lead + (self.n, NBR_K)),
            _ptr(nbr_rel, "nbr_rel", torch.float32, lead + (self.n, NBR_K * NBR_FEAT)), _stream(stream)))

    def rollout_graph(self, state, actions, action_type: int, n_substeps: int, K: int, obs_mode: int = OBS_NONE,
                      kin=None, nbr_idx=None, nbr_rel=None) -> "Graph":
        """A CUDA graph replaying rollout() with these buffers (mdg_rollout_graph_create)."""
        torch = _torch()
        per_step = actions.dim() == 3
        shape = (K, self.n, 4) if per_step else (self.n, 4)
        lead = (K,) if obs_mode == OBS_EVERY_STEP else ()
        g = ctypes.c_void_p()
        _check(lib().mdg_rollout_graph_create(
            self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
            _ptr(actions, "actions", torch.float32, shape), int(per_step), int(action_type), int(n_substeps), int(K),
            int(obs_mode), _ptr(kin, "kin", torch.float32, lead + (self.n, KIN_DIM)),
            _ptr(nbr_idx, "nbr_idx", torch.int32, lead + (self.n, NBR_K)),
            _ptr(nbr_rel, "nbr_rel", torch.float32, lead + (self.n, NBR_K * NBR_FEAT)), ctypes.byref(g)))
        return Graph(g, keep=(state, actions, kin, nbr_idx, nbr_rel))

    def autotune(self, state, actions, action_type: int, n_substeps: int = 5, K: int = 0, stream=None):
        """Time every block size on these inputs and keep the fastest (mdg_autotune).
        Returns (block size, mean ms)."""
        torch = _torch()
        per_step = actions.dim() == 3
        best = ctypes.c_int32()
        ms = ctypes.c_float()
        _check(lib().mdg_autotune(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                                  _ptr(actions, "actions", torch.float32), int(per_step), int(action_type),
                                  int(n_substeps), int(K), _stream(stream), ctypes.byref(best), ctypes.byref(ms)))
        return best.value, ms.value

    def features(self, state, rpm, raw, stream=None):
        """Raw surrogate inputs [n, 41] of the current state with the given RPMs (mdg_features)."""
        torch = _torch()
        _check(lib().mdg_features(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                                  _ptr(rpm, "rpm", torch.float32, (self.n, 4)),
                                  _ptr(raw, "raw", torch.float32, (self.n, MLP_IN)), _stream(stream)))

    def transition(self, state, rpm, applied, raw, delta, rpm_scale=None, n_substeps: int = 5, stream=None):
        """One transition of the plain integrator (mdg_transition): applied [n, 4] = rpm
        (times rpm_scale), raw [n, 41] the inputs of the state with them, one control step,
        delta [n, 13] the state change."""
        torch = _torch()
        _check(lib().mdg_transition(self._h, _ptr(state, "state", torch.float32, (STATE_PLANES, self.n, 4)),
                                    _ptr(rpm, "rpm", torch.float32, (self.n, 4)),
                                    _ptr(rpm_scale, "rpm_scale", torch.float32, (self.n, 4)),
                                    _ptr(applied, "applied", torch.float32, (self.n, 4)),
                                    _ptr(raw, "raw", torch.float32, (self.n, MLP_IN)),
                                    _ptr(delta, "delta", torch.float32, (self.n, MLP_OUT)), int(n_substeps),
                                    _stream(stream)))

    # -- output buffers
    def new_obs(self, device="cuda"):
        torch = _torch()
        return (torch.empty((self.n, KIN_DIM), dtype=torch.float32, device=device),
                torch.empty((self.n, NBR_K), dtype=torch.int32, device=device),
                torch.empty((self.n, NBR_K * NBR_FEAT), dtype=torch.float32, device=device))


# ---------------------------------------------------------------- learned surrogate
def mlp_flatten(layers) -> np.ndarray:
    """[(W [out, in], b [out]), ...] (padded shapes of MLP_DIMS) -> flat float32 parameters."""
    parts = []
    for W, b in layers:
        parts += [np.asarray(W, np.float32).reshape(-1), np.asarray(b, np.float32).reshape(-1)]
    flat = np.concatenate(parts)
    if flat.size != MLP_PARAMS:
        raise ValueError(f"expected {MLP_PARAMS} parameters, got {flat.size}")
    return flat


def mlp_unflatten(flat):
    """Flat parameters -> [(W [out, in], b [out]), ...]."""
    flat = np.asarray(flat)
    out, off = [], 0
    for fi, fo in zip(MLP_DIMS[:-1], MLP_DIMS[1:]):
        W = flat[off:off + fi * fo].reshape(fo, fi)
        off += fi * fo
        b = flat[off:off + fo]
        off += fo
        out.append((W, b))
    return out


class MLP:
    """The surrogate network (mdg_mlp): FP32 master parameters, bf16 copies, Adam state and
    scratch for batches of up to max_batch rows (a multiple of 128)."""

    def __init__(self, max_batch: int, init=None):
        flat = None if init is None else np.ascontiguousarray(
            mlp_flatten(init) if isinstance(init, (list, tuple)) else init, np.float32)
        self._m = ctypes.c_void_p()
        _check(lib().mdg_mlp_create(int(max_batch), None if flat is None else flat.ctypes.data_as(_VP),
                                    ctypes.byref(self._m)))
        self.max_batch = int(max_batch)

    def close(self):
        if self._m:
            lib().mdg_mlp_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        _check(lib().mdg_mlp_get_params(self._m, out.ctypes.data_as(_VP)))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        _check(lib().mdg_mlp_set_params(self._m, flat.ctypes.data_as(_VP)))

    def grads(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        _check(lib().mdg_mlp_get_grads(self._m, out.ctypes.data_as(_VP)))
        return out

    def set_normalization(self, in_mean, in_std, out_mean, out_std, in_lo, in_hi):
        arrs = [np.ascontiguousarray(a, np.float32) for a in (in_mean, in_std, out_mean, out_std, in_lo, in_hi)]
        _check(lib().mdg_mlp_set_normalization(self._m, *[a.ctypes.data_as(_VP) for a in arrs]))

    def fit_normalization(self, raw, delta, x_out, t_out, trim_frac: float = 0.005, margin: float = 0.1,
                          ood_z: float = 4.0, target_clip: float = 8.0, stream=None):
        """Standardise a set of transitions for training and set the normalisation from it
        (mdg_mlp_fit_normalization). Returns (finite rows, rows written to x_out / t_out)."""
        torch = _torch()
        N = raw.shape[0]
        n_fin, n_kept = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mdg_mlp_fit_normalization(
            self._m, _ptr(raw, "raw", torch.float32, (N, MLP_IN)), _ptr(delta, "delta", torch.float32, (N, MLP_OUT)),
            int(N), ctypes.c_float(trim_frac), ctypes.c_float(margin), ctypes.c_float(ood_z),
            ctypes.c_float(target_clip), _ptr(x_out, "x_out", torch.bfloat16, (N, MLP_IN_PAD)),
            _ptr(t_out, "t_out", torch.float32, (N, MLP_OUT_PAD)), ctypes.byref(n_fin), ctypes.byref(n_kept),
            _stream(stream)))
        return n_fin.value, n_kept.value

    def normalization(self):
        """(in_mean, in_std, out_mean, out_std, in_lo, in_hi) in use (mdg_mlp_get_normalization)."""
        arrs = [np.zeros(n, np.float32) for n in (MLP_IN, MLP_IN, MLP_OUT, MLP_OUT, MLP_IN, MLP_IN)]
        _check(lib().mdg_mlp_get_normalization(self._m, *[a.ctypes.data_as(_VP) for a in arrs]))
        return tuple(arrs)

    def standardize(self, raw, x, stream=None):
        torch = _torch()
        rows = raw.shape[0]
        _check(lib().mdg_mlp_standardize(self._m, _ptr(raw, "raw", torch.float32, (rows, MLP_IN)),
                                         _ptr(x, "x", torch.bfloat16, (rows, MLP_IN_PAD)), int(rows),
                                         _stream(stream)))

    def forward(self, x, y, stream=None):
        torch = _torch()
        B = x.shape[0]
        _check(lib().mdg_mlp_forward(self._m, _ptr(x, "x", torch.bfloat16, (B, MLP_IN_PAD)),
                                     _ptr(y, "y", torch.float32, (B, MLP_OUT_PAD)), int(B), _stream(stream)))

    def grad(self, x, t, loss=None, stream=None):
        torch = _torch()
        B = x.shape[0]
        _check(lib().mdg_mlp_grad(self._m, _ptr(x, "x", torch.bfloat16, (B, MLP_IN_PAD)),
                                  _ptr(t, "t", torch.float32, (B, MLP_OUT_PAD)), int(B),
                                  _ptr(loss, "loss", torch.float32, (1,)), _stream(stream)))

    def set_path(self, path: int):
        """Inference path: MLP_PATH_TCGEN05_PAIRS (default: the fused tensor-memory kernel with
        two tiles in flight per block), MLP_PATH_TCGEN05 (one tile per block) or
        MLP_PATH_MMA_SYNC."""
        _check(lib().mdg_mlp_set_path(self._m, int(path)))

    def set_train_path(self, path: int):
        """GEMMs of mdg_mlp_grad: MLP_PATH_TCGEN05 (default) or MLP_PATH_MMA_SYNC."""
        _check(lib().mdg_mlp_set_train_path(self._m, int(path)))

    def set_wait_limits(self, try_waits: int = -1, polls: int = -1):
        """Bounds of the tcgen05 kernel's mbarrier waits (negative: the defaults)."""
        _check(lib().mdg_mlp_set_wait_limits(self._m, int(try_waits), int(polls)))

    def status(self, stream=None) -> int:
        bits = ctypes.c_uint32()
        _check(lib().mdg_mlp_status(self._m, _stream(stream), ctypes.byref(bits)))
        return bits.value

    def adam(self, lr: float, stream=None):
        _check(lib().mdg_mlp_adam(self._m, ctypes.c_float(lr), _stream(stream)))

    def step(self, handle: "Handle", state, action, action_type: int, n_substeps: int = 5, ood_z: float = 4.0,
             n_fallback=None, stream=None):
        """One control step with the surrogate (mdg_surrogate_step)."""
        torch = _torch()
        _check(lib().mdg_surrogate_step(handle._h, self._m,
                                        _ptr(state, "state", torch.float32, (STATE_PLANES, handle.n, 4)),
                                        _ptr(action, "action", torch.float32, (handle.n, 4)), int(action_type),
                                        int(n_substeps), ctypes.c_float(ood_z),
                                        _ptr(n_fallback, "n_fallback", torch.int32, (1,)), _stream(stream)))
