"""Benchmark of the batched multi-drone dynamics step on GB300.

One benchmark step is one control step of the whole hot path over the full-aero swarm
(16384 environments x 4 Crazyflies = 65536 drones): the PID waypoint controller, 5
physics substeps at 240 Hz with motor model, ground effect, drag and pairwise downwash,
and the KIN + 4-neighbour observations -- one launch of the fused step kernel through
the C ABI (mdg_step_obs). The metric is drone-substeps per second.

Timing: W untimed warm-up steps, then K timed steps back to back with inputs larger than
L2: 16 independent swarms of the full size, each with its own state, waypoints and
observation buffers, are stepped in rotation (one CUDA graph holds one step of every swarm
and is replayed), so each step's data was last touched 15 steps and ~300 MB earlier, well
beyond the 129 MB L2; CUDA events on the launching stream bracket the whole region, with a
barrier and a synchronisation on both sides. Each swarm is reset to its initial state
before a region (outside it); a region holds at most one 1000-step episode per swarm.
Under torchrun each rank runs its own swarms on its own GPU (environments are independent:
weak scaling, no data-path collective); the time is the max over ranks.

Also reported, on swarm 0: the same step isolated (the L2 flushed before every step -- a
512 MiB buffer written, then read back -- and every step bracketed by its own events, so
one launch's latency is counted per step), an end-to-end number through the public API
with host buffers (waypoints read and observations written in pinned host memory every
step, synchronised every step), the 1000-step episode as one persistent launch, the
roofline of the step kernel against the measured HBM bandwidth, SM clocks sampled during
the timed region, and the FP64 oracle timed on the host cores on a bounded sample.

--model / --integrator / --gnd-heights select the drone model (CF2X, CF2P, RACE), Euler or
RK4 substeps and the ground-effect heights (centre of mass, or per rotor) for the dynamics
workloads; the defaults are the headline configuration (CF2X, Euler, centre of mass).

--impl reference times the oracle alone (the reference arm of this project).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "drone-substeps/s on 1 GB300 (FP32 vs oracle)"
UNIT = "drone-substeps/s"
N_SUB = 5
EPISODE = 1000
# Algorithmic bytes per drone and control step (the count the roofline divides by): the
# 13-value state read and written, the controller's 6 integrals read and written where its
# loops run, the action, the observations. The kernel moves 24 B more per drone than this
# count on the PID workload: the padding lane of the integral plane (read and written) and
# the a_{t-1} plane (written; KIN carries the same four RPMs).
STATE_BYTES = 13 * 4
INTEG_BYTES = 6 * 4
ACTION_BYTES = 16
OBS_BYTES = 80 + 16 + 96  # KIN, neighbour indices, neighbour features
BYTES_PER_DRONE_STEP = 2 * STATE_BYTES + 2 * INTEG_BYTES + ACTION_BYTES + OBS_BYTES  # 360
# A bounded device sleep enqueued before the start event of a back-to-back region, so that
# the host has submitted the region's launches before the GPU reaches the first one and the
# events measure device time, not host submission (about 0.2 ms at 2 GHz).
HEAD_START_CYCLES = 400_000

# DRAM traffic of one step-kernel launch on the full-aero workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel source whose
# sha256 prefix is recorded with it; profiles/ holds the capture's summary.
NCU_TRAFFIC = {"kernel_sha": "cf5d9e7547c2a1c2", "bytes": 6319104 + 0}


def kernel_sha() -> str:
    with open(os.path.join(ROOT, "paper_2606_08039_gb300", "csrc", "mdg_step.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


ACTION_CHOICES = {"pid": 1, "rpm": 0, "rpm_norm": 3, "one_d_rpm": 4, "vel": 5, "attitude": 6, "mixed": 2}


DR_DEPTH = 3   # action-history depth of the randomized workload (latency up to 2 control steps)
DR_SEED = 5    # wind draws of the randomized workload


def model_config(args) -> dict:
    out = {"model": args.model, "integrator": args.integrator, "gnd_heights": args.gnd_heights,
           "actions": getattr(args, "actions", "pid"), "controller": getattr(args, "controller", "pid")}
    if getattr(args, "randomize", False):
        out["randomization"] = ("recommended-ranges rows per environment, motor lag, action latency "
                                f"(history depth {DR_DEPTH}), COMBINED wind")
    return out


def is_default_model(args) -> bool:
    return ((args.model, args.integrator, args.gnd_heights) == ("cf2x", "euler", "com")
            and getattr(args, "actions", "pid") == "pid" and getattr(args, "controller", "pid") == "pid"
            and not getattr(args, "randomize", False))


def action_types(args, n_envs: int, seed: int) -> np.ndarray:
    """uint8 [n_envs] per-environment action types of the full-aero workload."""
    from paper_2606_08039_gb300 import workloads as wl
    if args.actions == "mixed":
        return wl.all_action_types(seed, n_envs)
    return np.full(n_envs, ACTION_CHOICES[args.actions], np.uint8)


def library_constants(args):
    """The library's constants for the chosen model, integrator and ground-effect heights."""
    import paper_2606_08039_gb300 as mdg
    c = getattr(mdg.Constants, args.model)()
    c.integrator = mdg.INTEGRATOR_RK4 if args.integrator == "rk4" else mdg.INTEGRATOR_EULER
    c.gnd_heights = mdg.GND_ROTOR if args.gnd_heights == "rotor" else mdg.GND_COM
    if getattr(args, "controller", "pid") == "dsl":
        c = c.with_dsl()
    return c


def oracle_params(args):
    """The oracle's own parameters for the same choice (CPU-baseline and reference legs)."""
    import oracle
    P = getattr(oracle, args.model)()
    P.integrator = oracle.RK4 if args.integrator == "rk4" else oracle.EULER
    P.gnd_heights = oracle.GND_ROTOR if args.gnd_heights == "rotor" else oracle.GND_COM
    if getattr(args, "controller", "pid") == "dsl":
        P = oracle.controller_dsl(P)
    return P


def oracle_workload(args, sw, seed: int):
    """(env action types, actions [1, n, 4] float64, setpoints or None) of the full-aero
    workload for the oracle legs."""
    from paper_2606_08039_gb300 import workloads as wl
    P = oracle_params(args)
    types = action_types(args, sw.n_envs, seed)
    if args.actions == "pid":
        act = wl.waypoints(seed, sw.n)
    else:
        act = wl.typed_actions(sw.drones_per_env, types, seed, 0, oracle_hover(P), P.mass * P.g)
    sp = np.full((sw.n, 4), np.nan) if args.controller == "dsl" else None
    dr = None
    if getattr(args, "randomize", False):
        import oracle
        dr = oracle.Randomization(sw.n_envs, sw.n, DR_DEPTH, DR_SEED)
        dr.env_dr[:] = wl.dr_table(seed, sw.n_envs, depth=DR_DEPTH).astype(np.float64)
    return types.astype(np.int32), act.astype(np.float64)[None], sp, dr


def oracle_hover(P) -> float:
    import oracle
    return oracle.hover_rpm(P)


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", 1700.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, windows=None) -> dict:
        """Median SM clock, maximum clock and throttle reasons over the samples read inside
        `windows` (host perf_counter intervals of the timed region; all samples if none fall
        inside)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        lines = self.lines
        if windows:
            inside = [(t, l) for t, l in lines if any(a <= t <= b + 0.06 for a, b in windows)]
            if inside:
                lines = inside
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "timed region" if windows and lines is not self.lines else "whole run"}


def replica_seed(rank: int) -> int:
    """Each rank simulates its own independent full-aero swarm (weak scaling)."""
    return 1 + rank


def combine_over_ranks(times_ms, world: int, device=None):
    """Max over ranks of each timed quantity (a barrier-bracketed region is as slow as its
    slowest rank). Uses the default process group when world > 1."""
    import torch
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def throughput(units_per_step_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job units per second: every rank's units over the max-over-ranks time."""
    return units_per_step_per_rank * world * steps / (total_ms * 1e-3)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleShards:
    """The full-aero swarm's oracle inputs split into `n_shards` contiguous environment
    ranges, one per host thread. The environments are independent, so each range runs the
    oracle's own control-step routine, unchanged, on its own slice and its own buffers
    (oracle.control_steps_into: no copies per call); ctypes releases the GIL for the
    duration of the C call, so the threads run on separate cores. Neighbour indices and the
    randomization's counters are shard-relative (the values differ from one unsharded call,
    the work does not)."""

    def __init__(self, args, sw, seed: int, n_shards: int):
        import oracle
        self.oracle = oracle
        self.P = oracle_params(args)
        acts, wp, sp, dr = oracle_workload(args, sw, seed)
        x, flags = sw.x13(), sw.flags.astype(np.int32)
        bounds = np.linspace(0, sw.n_envs, max(1, min(n_shards, sw.n_envs)) + 1).astype(int)
        self.shards = []
        for e0, e1 in zip(bounds[:-1], bounds[1:]):
            d0, d1 = int(sw.env_off[e0]), int(sw.env_off[e1])
            sh = {"off": (sw.env_off[e0:e1 + 1] - d0).astype(np.int32), "flags": flags[e0:e1].copy(),
                  "acts": acts[e0:e1].copy(), "x": x[d0:d1].astype(np.float64), "integ": np.zeros((d1 - d0, 6)),
                  "a": np.zeros((d1 - d0, 4)), "wp": np.ascontiguousarray(wp[:, d0:d1], dtype=np.float64),
                  "sp": None if sp is None else sp[d0:d1].copy(), "dr": None,
                  "kin": np.zeros((d1 - d0, 20)), "idx": np.zeros((d1 - d0, 4), np.int32),
                  "rel": np.zeros((d1 - d0, 24))}
            if dr is not None:
                r = oracle.Randomization(e1 - e0, d1 - d0, dr.hist.shape[0], dr.seed)
                r.env_dr[:] = dr.env_dr[e0:e1]
                sh["dr"] = r
            self.shards.append(sh)
        self.n = sw.n

    def _run(self, sh):
        self.oracle.control_steps_into(self.P, sh["off"], sh["flags"], sh["acts"], sh["x"], sh["integ"], sh["a"],
                                       sh["wp"], N_SUB, sh["kin"], sh["idx"], sh["rel"], setpoint=sh["sp"],
                                       dr=sh["dr"])

    def step(self, pool) -> None:
        """One control step (PID + substeps + observations) of every shard."""
        if pool is None:
            for sh in self.shards:
                self._run(sh)
        else:
            list(pool.map(self._run, self.shards))


def cpu_baseline(args, seconds_target: float = 10.0, all_cores_seconds: float = 5.0) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the full-aero workload: the
    full 16384 x 4 swarm for as many control steps (PID + 5 substeps + observations each)
    as fit in about the given seconds, on every host core (the environments split into one
    range per thread) and on one host core, with the chosen model. The all-cores figure is
    the reported value."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2606_08039_gb300 import workloads as wl
    sw = wl.full_aero(1)

    def timed(n_threads: int, budget: float):
        shards = OracleShards(args, sw, 1, n_threads)
        pool = ThreadPoolExecutor(n_threads) if n_threads > 1 else None
        try:
            steps = 0
            t0 = time.perf_counter()
            while True:
                shards.step(pool)
                steps += 1
                dt = time.perf_counter() - t0
                if dt >= budget or steps >= 200:
                    return sw.n * N_SUB * steps / dt, steps, dt
        finally:
            if pool is not None:
                pool.shutdown()

    cores = host_cores()
    v1, s1, t1 = timed(1, seconds_target)
    single = {"value": v1, "cores": 1,
              "sample": f"{s1} control steps of the whole swarm, single thread ({t1:.1f} s)"}
    if cores > 1:
        vc, sc, tc = timed(cores, all_cores_seconds)
    else:
        vc, sc, tc = v1, s1, t1
    return {"value": vc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full-aero swarm 16384 envs x 4 drones, {sc} control steps x {N_SUB} substeps with PID and "
                      f"observations, FP64, environments split over {cores} threads ({tc:.1f} s)",
            "single_core": single, **model_config(args)}


def run_reference(args) -> None:
    """Reference arm: the FP64 oracle timed as it stands on the host cores (the environments
    split into one range per thread), on a bounded sample of the same workload per step
    (one control step of a subset of the swarm's environments, sized so that the whole run
    takes about a minute)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    from paper_2606_08039_gb300 import workloads as wl
    cores = host_cores()
    # about a minute of host work for the whole run: 2048 environments per core for 5000
    # steps, fewer per step for more steps (multiples of 64, at most the whole swarm, at
    # least 4096 so that the threads' per-step overhead stays small)
    n_envs = int(min(16384, max(4096, round(2048 * cores * 5000 / max(1, args.steps + args.warmup) / 64) * 64)))
    sw = wl.full_aero(1, n_envs=n_envs)
    shards = OracleShards(args, sw, 1, cores)
    pool = ThreadPoolExecutor(cores) if cores > 1 else None
    try:
        for _ in range(args.warmup):
            shards.step(pool)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            shards.step(pool)
        dt = time.perf_counter() - t0
    finally:
        if pool is not None:
            pool.shutdown()
    value = sw.n * N_SUB * args.steps / dt
    sample = (f"per step: {n_envs} envs x 4 drones of the full-aero swarm, one control step (PID + {N_SUB} "
              f"substeps + observations), FP64 oracle, environments split over {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"full_aero 16384 envs x 4 drones (sampled {n_envs} envs per step)", "n_substeps": N_SUB,
                   "l2": "n/a (host)", **model_config(args)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# FP32 arithmetic per drone and substep, counted from the oracle's operation list (an FMA
# counts as 2 flops, a special-function evaluation as 1): the explicit integrator with
# thrust, gravity, Newton-Euler, exponential map and Euler update; each optional effect;
# per other drone of the environment the downwash pair test, and per drone above it the
# pair term. PID and observations are counted per control step.
FLOPS_BASE, FLOPS_GND, FLOPS_DRAG = 130, 8, 16
FLOPS_DW_PAIR_TEST, FLOPS_DW_PAIR_TERM = 8, 16
FLOPS_PID, FLOPS_OBS, FLOPS_OBS_PER_NEIGHBOUR = 150, 60, 8
# RK4 (same counting): per stage the quaternion normalisation (12), the body z axis (9),
# thrust and gravity (4), Newton-Euler (18), q' = 1/2 q (x) [0, w] (24), v' (3) and the stage
# update of the 13 components (sum and next stage state, 52); per substep the final update
# and renormalisation (38). Each effect is evaluated once per stage.
FLOPS_RK4_STAGE, FLOPS_RK4_FINAL = 122, 38
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock = 80.5
ALU_PEAK_SRC = "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz"


def algorithmic_flops(sw, K: int, n_sub: int, obs_steps: int, pid_mask=None, rk4: bool = False) -> float:
    """Counted FP32 flops of K control steps of a swarm (pairs above: half the others)."""
    N = sw.drones_per_env.astype(np.float64)
    f = sw.flags
    effects = ((f & 1) > 0) * FLOPS_GND + ((f & 2) > 0) * FLOPS_DRAG
    effects = effects + ((f & 4) > 0) * ((N - 1) * FLOPS_DW_PAIR_TEST + 0.5 * (N - 1) * FLOPS_DW_PAIR_TERM)
    per_sub = (4 * (FLOPS_RK4_STAGE + effects) + FLOPS_RK4_FINAL) if rk4 else FLOPS_BASE + effects
    pid = np.zeros_like(N) if pid_mask is None else pid_mask.astype(np.float64) * FLOPS_PID
    per_step = n_sub * per_sub + pid
    total = np.sum(N * (K * per_step + obs_steps * (FLOPS_OBS + FLOPS_OBS_PER_NEIGHBOUR * (N - 1))))
    return float(total)


def algorithmic_bytes(sw, types, act_type: int, dsl: bool, dr_depth: int = 0) -> int:
    """Bytes one fused control step must move for the full-aero workload: per drone the
    13-value state read and written (52 + 52 B), the action (16 B), the observations (192 B),
    the controller's 6 integrals read and written (24 + 24 B) where its loops run (PID, VEL,
    ATTITUDE), and with the DSL controller the setpoint of each waypoint-driven drone read and
    written (32 B). 360 B for PID actions, 312 B for RPM actions. Under randomization (history
    depth D): the rotor speeds read and written (32 B), the action history shifted (D - 1
    reads, D writes of 16 B), and per environment its 128 B row and its 32 B wind state read
    and written."""
    per_env = np.full(sw.n_envs, 2 * STATE_BYTES + ACTION_BYTES + OBS_BYTES, np.int64)
    per_env += 2 * INTEG_BYTES * np.isin(types, (1, 5, 6))
    if dsl:
        per_env += 32 * (types == 1)
    total = int(np.sum(per_env * sw.drones_per_env))
    if dr_depth:
        total += sw.n * (32 + 16 * (2 * dr_depth - 1)) + sw.n_envs * (128 + 64)
    return total


def binding_roofline(bytes_launch: float, flops_launch: float, sec: float, peaks) -> dict:
    """The roofline of a launch against the bound whose ideal time is the longer: HBM
    (algorithmic bytes over the measured copy bandwidth) or FP32 ALU (counted flops over
    the derived peak); the other bound is reported beside it."""
    t_hbm = bytes_launch / (peaks["hbm_gbs"] * 1e9)
    t_alu = flops_launch / (FP32_PEAK_TFLOPS * 1e12)
    hbm = {"bound": "hbm", "achieved": bytes_launch / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "peak_src": peaks["src"], "algorithmic_bytes_per_launch": bytes_launch}
    alu = {"bound": "alu", "achieved": flops_launch / sec / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
           "peak_src": ALU_PEAK_SRC, "algorithmic_flops_per_launch": flops_launch}
    for r in (hbm, alu):
        r["frac"] = r["achieved"] / r["peak"]
    main, other = (hbm, alu) if t_hbm >= t_alu else (alu, hbm)
    main["other_bound"] = {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    return main


EPISODE_REPS = 3
N_SWARMS = 16            # independent full-size swarms stepped in rotation in the timed region
SWARM_SEED_STRIDE = 97   # seed of swarm k: the rank's replica seed + 97 k
SWARM_BYTES = 65536 * (96 + 16 + 80 + 16 + 96)  # per swarm and step: state planes, waypoints, KIN, indices, features
ISOLATED_STEPS = 1000    # steps of the isolated (flushed, per-step events) measurement
# algorithmic bytes of a K-step rollout with observations every step: the state and the
# integrals read and written once (2 x (52 + 24) B), the waypoint once (16 B), KIN + indices
# + features every step
BYTES_OBS_PER_DRONE_STEP = OBS_BYTES


def nonfinite_fraction(states) -> float:
    """Fraction of drones whose position, quaternion, velocity or body rate (state planes
    0-3) is not finite, over the given [6, n, 4] state tensors."""
    import torch
    bad = sum(int((~torch.isfinite(st[0:4]).all(dim=2).all(dim=0)).sum()) for st in states)
    return bad / sum(int(st.shape[1]) for st in states)


def episode_line(n: int, world: int, ep_ms: float, peaks, flops_step: float, episode: int = EPISODE) -> dict:
    value = throughput(n * N_SUB * episode, world, EPISODE_REPS, ep_ms)
    sec = ep_ms / EPISODE_REPS * 1e-3
    nbytes = n * (2 * (STATE_BYTES + INTEG_BYTES) + ACTION_BYTES + episode * BYTES_OBS_PER_DRONE_STEP)
    roof = binding_roofline(nbytes, flops_step * episode, sec, peaks)
    roof["kernel"] = "rollout_kernel<obs every step>"
    return {"what": f"the {episode}-control-step episode as one persistent rollout per launch (mdg_rollout, "
                    "observations of every step written), L2 flushed between episodes; the headline value "
                    "above is one control step per launch",
            "value": value, "unit": UNIT, "ms_per_episode": ep_ms / EPISODE_REPS, "episodes": EPISODE_REPS,
            "us_per_control_step": ep_ms / EPISODE_REPS / episode * 1e3,
            "roofline": roof}


def uneven_vs_uniform(sw, acts, c, K: int, dev, timed) -> dict:
    """The uneven batch's control steps run as uniform batches: its environments grouped by
    (size, physics subset, action type), each group a handle of its own (one environment size
    and physics subset: the compile-time kernel variants where one exists), its K-step rollout
    autotuned (block size, schedule, item size) and captured as a CUDA graph. One step = every
    group's graph in turn, observations after the last step; the state of every group reset
    before each step (untimed)."""
    import torch
    import paper_2606_08039_gb300 as mdg
    env_off = sw.env_off
    groups = {}
    for e in range(sw.n_envs):
        key = (int(sw.drones_per_env[e]), int(sw.flags[e]), int(sw.act_type[e]))
        if key[0] > 0:
            groups.setdefault(key, []).append(e)
    runs = []
    acts_np = acts.cpu().numpy()
    for (N, fl, at), envs in sorted(groups.items()):
        idx = np.concatenate([np.arange(env_off[e], env_off[e + 1]) for e in envs])
        h = mdg.Handle(np.full(len(envs), N, np.int32), np.full(len(envs), fl, np.uint32), c)
        init = mdg.pack_state(sw.p[idx], sw.q[idx], sw.v[idx], sw.w[idx], device=dev)
        st = init.clone()
        a = torch.as_tensor(np.ascontiguousarray(acts_np[:, idx]), device=dev)
        kin, nidx, rel = h.new_obs(dev)
        h.autotune(st, a, at, N_SUB, K)
        g = h.rollout_graph(st, a, at, N_SUB, K, mdg.OBS_LAST, kin, nidx, rel)
        runs.append((h, init, st, a, (kin, nidx, rel), g))

    def step_all():
        for r in runs:
            r[5].launch()

    def reset_all():
        for r in runs:
            r[2].copy_(r[1])
    timed(step_all, 3, reset_all)
    n = 50
    ms = timed(step_all, n, reset_all) / n
    for r in runs:
        r[5].close()
    return {"what": "the same environments and actions as uniform batches grouped by (size, physics subset, action "
                    "type), each group's K-step rollout autotuned and replayed as its own CUDA graph, the groups in turn",
            "groups": len(runs), "ms_per_step": ms, "value": sw.n * N_SUB * K / (ms * 1e-3)}


def run_other(args) -> None:
    """The other swarms, on one GPU:
    uneven  4096 envs of 1..32 drones, mixed physics subsets and RPM/PID actions: one
            step = one replay of the CUDA graph of a 32-control-step persistent rollout
            (observations after the last step), block size autotuned; state reset to the
            initial swarm before every replay (untimed).
    dense   1024 envs x 64 drones, all effects, RPM actions: one step = one control step
            (mdg_step_obs), 16 action sets cycled.
    single  64 envs x 1 drone, ground effect + drag: one step = the 240-control-step
            episode in one rollout launch (latency-bound; also reported per control step)."""
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)
    c = library_constants(args)
    hover = c.hover_rpm()
    extra = {}
    if args.workload == "uneven":
        sw, K, obs_steps = wl.uneven(2), 32, 1
        h = mdg.Handle(sw.drones_per_env, sw.flags, c)
        h.set_action_types(sw.act_type)
        acts = torch.as_tensor(np.stack([wl.mixed_actions(sw, 2, k, hover) for k in range(K)]), device=dev)
        init = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
        state = init.clone()
        kin, idx, rel = h.new_obs(dev)
        block, _ = h.autotune(state, acts, mdg.ACT_MIXED, N_SUB, K)
        sched_mode, item_cap = h.rollout_schedule
        extra["autotuned"] = {"block": block, "schedule": ["dynamic", "static"][sched_mode], "item_drones": item_cap}
        graph = h.rollout_graph(state, acts, mdg.ACT_MIXED, N_SUB, K, mdg.OBS_LAST, kin, idx, rel)

        def run():
            graph.launch(stream)
        reset = True
        pid_mask = sw.act_type == mdg.ACT_PID
        substeps = sw.n * N_SUB * K
        desc = (f"uneven: 4096 envs, N in {{1,2,4,8,16,32}} ({sw.n} drones), 8 physics subsets, RPM/PID mixed; "
                f"one step = CUDA-graph replay of a {K}-control-step persistent rollout, obs after the last")
        launches = 1
        # the same 32 control steps as 32 single-step launches, for comparison
        extra_fn = lambda: [h.step_obs(state, acts[k], mdg.ACT_MIXED, N_SUB, kin, idx, rel, stream=stream)
                            for k in range(K)]
    elif args.workload == "dense":
        sw, K, obs_steps = wl.dense(5), 1, 1
        h = mdg.Handle(sw.drones_per_env, sw.flags, c)
        acts = [torch.as_tensor(wl.rpm_actions(5, sw.n, k, hover), device=dev) for k in range(16)]
        init = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
        state = init.clone()
        kin, idx, rel = h.new_obs(dev)
        block = h.block_size
        counter = [0]

        def run():
            if counter[0] and counter[0] % 500 == 0:  # 500-step episodes
                state.copy_(init)
            h.step_obs(state, acts[counter[0] % 16], mdg.ACT_RPM, N_SUB, kin, idx, rel, stream=stream)
            counter[0] += 1
        reset = False
        pid_mask = None
        substeps = sw.n * N_SUB
        desc = "dense: 1024 envs x 64 drones, all effects, RPM actions; one step = one control step (mdg_step_obs)"
        launches = 1
        extra_fn = None
    else:
        sw, K, obs_steps = wl.single(0), 240, 1
        h = mdg.Handle(sw.drones_per_env, sw.flags, c)
        acts = torch.as_tensor(np.stack([wl.rpm_actions(0, sw.n, k, hover) for k in range(K)]), device=dev)
        init = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
        state = init.clone()
        kin, idx, rel = h.new_obs(dev)
        block = h.block_size

        def run():
            h.rollout(state, acts, mdg.ACT_RPM, N_SUB, K, mdg.OBS_LAST, kin, idx, rel, stream=stream)
        reset = True
        pid_mask = None
        substeps = sw.n * N_SUB * K
        desc = "single: 64 envs x 1 drone, ground effect + drag, RPM actions; one step = the 240-step episode in one rollout"
        launches = 1
        extra_fn = None

    def flush_l2():
        flush.fill_(1.0)
        torch.sum(flush, dim=0, out=sink)

    def timed_each(fn, n, before=None):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for i in range(n):
            if before is not None:
                before()
            elif reset:
                state.copy_(init)
            flush_l2()
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in zip(st, en)]

    def timed(fn, n, before=None):
        return float(sum(timed_each(fn, n, before)))

    steps = min(args.steps, 2000)
    timed(run, args.warmup)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    per_step = timed_each(run, steps)
    total_ms = float(sum(per_step))
    clk = clocks.stop()
    extra["ms_per_step_spread"] = {"min": min(per_step), "median": statistics.median(per_step),
                                   "max": max(per_step)}
    rc, bits, _ = h.status()
    nonfinite_frac = nonfinite_fraction([state])
    if extra_fn is not None:
        timed(extra_fn, 3)
        per_step_ms = timed(extra_fn, min(steps, 200)) / min(steps, 200)
        extra["same_work_as_single_step_launches"] = {"value": substeps / (per_step_ms * 1e-3), "ms": per_step_ms,
                                                      "launches": K}
    if args.workload == "uneven":
        extra["vs_best_uniform_kernels"] = uneven_vs_uniform(sw, acts, c, K, dev, timed)
    ms = total_ms / steps
    flops = algorithmic_flops(sw, K, N_SUB, obs_steps, pid_mask, rk4=args.integrator == "rk4")
    achieved = flops / (ms * 1e-3) / 1e12
    out = {
        "metric": METRIC, "value": substeps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "n_drones": sw.n, "control_steps_per_step": K, "n_substeps": N_SUB,
                   "block_size": block, "l2": "flushed between timed steps (512 MiB written, then read back)",
                   **model_config(args)},
        "gpu_launches": launches * steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "peak_src": ALU_PEAK_SRC, "algorithmic_flops_per_step": flops},
        "clocks": clk, "nonfinite_during_timing": bool(bits & mdg.STATUS_NONFINITE),
        "nonfinite_fraction_after_timing": nonfinite_frac,
    }
    if args.workload == "single":
        out["us_per_control_step"] = ms * 1e3 / K
    out.update(extra)
    print(json.dumps(out))


# Camera frames (mdg_render): the frames themselves (RGBA, depth and segment, 12 B per pixel)
# are the algorithmic bytes, and the roofline is HBM. The brute-force arithmetic, counted from
# the oracle's ray caster (ray generation 25 flops per pixel, ground 15, shading and outputs
# 30, and 30 per other drone of the environment), is reported beside it as an upper bound:
# the kernel tests a drone only where its screen rectangle covers the pixels.
FLOPS_PIXEL_BASE, FLOPS_PIXEL_PAIR = 70, 30
CAM_PIXELS = 48 * 64
CAM_BYTES_PER_FRAME = CAM_PIXELS * (4 + 4 + 4) + 32  # RGBA, depth, segment; the camera drone's pose


def run_camera(args) -> None:
    """Camera frames of the full-aero swarm (16384 envs x 4 drones): one step renders every
    drone's 48 x 64 RGBA, depth and segmentation frame (one mdg_render launch, 2.4 GB of
    frames), L2 flushed between steps."""
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sw = wl.full_aero(1, n_envs=args.envs or 16384)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
    rgba, depth, seg = h.new_frames(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def timed(n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in ev:
            flush.fill_(1.0)
            torch.sum(flush, dim=0, out=sink)
            a.record(stream)
            h.render(state, rgba, depth, seg, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in ev))

    steps = min(args.steps, 500)
    timed(args.warmup)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    total_ms = timed(steps)
    clk = clocks.stop()
    ms = total_ms / steps
    N = sw.drones_per_env.astype(np.float64)
    flops = float(np.sum(N * CAM_PIXELS * (FLOPS_PIXEL_BASE + FLOPS_PIXEL_PAIR * (N - 1))))
    nbytes = sw.n * CAM_BYTES_PER_FRAME
    peaks = measured_peaks()
    roof = binding_roofline(nbytes, 0.0, ms * 1e-3, peaks)
    roof.pop("other_bound", None)
    roof["brute_force_flops_per_launch"] = flops
    roof["kernel"] = "render_kernel"
    out = {
        "metric": "camera frames/s on 1 GB300 (48x64 RGBA + depth + segmentation, FP32 ray casting vs oracle)",
        "value": sw.n / (ms * 1e-3), "unit": "frames/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"camera: every drone of the full-aero swarm ({sw.n_envs} envs x 4), one mdg_render per step",
                   "n_frames": sw.n, "l2": "flushed between timed steps (512 MiB written, then read back)"},
        "pixels_per_s": sw.n * CAM_PIXELS / (ms * 1e-3),
        "gpu_launches": steps, "roofline": roof, "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = camera_cpu_baseline()
    print(json.dumps(out))


def camera_cpu_baseline(seconds_target: float = 10.0) -> dict:
    """The FP64 oracle's ray caster, as it stands, on the full-aero swarm's cameras, for as
    many frames as fit in about `seconds_target` seconds on one host core."""
    import oracle
    from oracle import camera
    from paper_2606_08039_gb300 import workloads as wl
    P = oracle.cf2x()
    sw = wl.full_aero(1, n_envs=4096)
    x = sw.x13()
    frames = 0
    t0 = time.perf_counter()
    while True:
        e, j = divmod(frames, 4)
        camera.render(P, x[4 * e:4 * e + 4], j, first_index=4 * e)
        frames += 1
        dt = time.perf_counter() - t0
        if dt >= seconds_target or frames >= 4 * 4096:
            break
    return {"value": frames / dt, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"{frames} frames of the full-aero swarm's cameras, FP64 numpy, single thread ({dt:.1f} s)"}


def run_mlp(args) -> None:
    """The surrogate network's inference kernels alone: 262144 rows (the 65536 x 4 swarm),
    initial weights, bf16 inputs; the fused tcgen05 kernel with two tiles in flight per block
    (the step's default path) and, for comparison, its single-tile form and the per-layer
    mma.sync GEMMs. Tensor roofline against the measured bf16 peak."""
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    rows = 262144
    m = mdg.MLP(rows, wl.mlp_init(3))
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    x = torch.randn((rows, mdg.MLP_IN_PAD), generator=g, device=dev).to(torch.bfloat16)
    y = torch.empty((rows, mdg.MLP_OUT_PAD), device=dev)
    flops = 2.0 * rows * (64 * 256 + 2 * 256 * 256 + 256 * 32)
    res = {}
    steps = min(args.steps, 500)
    for name, path in (("mma_sync", mdg.MLP_PATH_MMA_SYNC), ("tcgen05", mdg.MLP_PATH_TCGEN05),
                       ("tcgen05_pairs", mdg.MLP_PATH_TCGEN05_PAIRS)):
        m.set_path(path)
        for _ in range(args.warmup):
            m.forward(x, y, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            m.forward(x, y, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / steps
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    ach = flops / (res["tcgen05_pairs"] * 1e-3) / 1e12
    print(json.dumps({
        "per_path_ms": res,
        "metric": "surrogate network rows/s", "value": rows / (res["tcgen05_pairs"] * 1e-3), "unit": "rows/s",
        "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": res["tcgen05_pairs"],
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "surrogate network forward, 262144 rows, 64-256-256-256-32, bf16/FP32 accumulation",
                   "l2": "inputs (33.5 MB) and weights stay in L2 between launches"},
        "mma_sync_ms": res["mma_sync"], "gpu_launches": steps,
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_tflops"], "traffic": None, "peak_src": "measured (bf16 burst)",
                     "kernel": "mlp_umma_pair_kernel", "algorithmic_flops_per_launch": flops},
        "status": m.status()}))


def training_step_ms(data, steps: int = 200, batch: int = 8192) -> dict:
    """Milliseconds per training step (mdg_mlp_grad of one batch + mdg_mlp_adam) of each
    training path, on a fresh network and the same batches of the standardised data set."""
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import workloads as wl
    out = {}
    gen = torch.Generator(device=data.x.device)
    for name, path in (("tcgen05", mdg.MLP_PATH_TCGEN05), ("mma_sync", mdg.MLP_PATH_MMA_SYNC)):
        m = mdg.MLP(batch, wl.mlp_init(5))
        m.set_train_path(path)
        gen.manual_seed(0)
        idx = torch.randint(0, len(data), (steps + 5, batch), generator=gen, device=data.x.device)
        xs = [data.x.index_select(0, i) for i in idx]
        ts = [data.t.index_select(0, i) for i in idx]
        loss = torch.zeros(1, device=data.x.device)
        for k in range(5):
            m.grad(xs[k], ts[k], loss)
            m.adam(1e-3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k in range(5, steps + 5):
            m.grad(xs[k], ts[k], loss)
            m.adam(1e-3)
        b.record()
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(b) / steps
        del xs, ts
    return {"ms_per_step": out, "batch": batch, "steps": steps,
            "what": "one training step (forward, backward, Adam) of a batch of 8192 transitions per path"}


def run_surrogate(args) -> None:
    """The learned surrogate on one GPU: trained on ~10M transitions generated by the
    full-aero kernels (16384 envs x 4 drones, 153 control steps of PID with +-10% RPM
    perturbations), then one control step of 65536 envs x 4 drones (PID waypoints) with the
    surrogate (fused tcgen05 network, out-of-distribution environments on the plain
    integrator) against the plain fused step on the same swarm. Metric: drone-control-steps/s.
    Also: the one-step error of the surrogate against the plain integrator on the regular
    regime, the out-of-distribution fraction, and the tensor roofline of the network kernel."""
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import surrogate as sg
    from paper_2606_08039_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    raw, delta = sg.generate_transitions(16384, 153, seed=3, device=dev)
    data = sg.Dataset(raw, delta)
    del raw, delta
    sw = wl.surrogate_eval(4, 65536)
    m = mdg.MLP(sw.n, wl.mlp_init(3))
    data.attach(m)
    hist = sg.fit(m, data, epochs=4, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_train = len(data)
    kept = data.kept_fraction
    out_std = data.out_std
    out_mean = data.out_mean
    train_paths = training_step_ms(data)
    del data

    h = mdg.Handle(sw.drones_per_env, sw.flags)
    init = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
    wp = torch.as_tensor(wl.waypoints(4, sw.n), device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def timed(fn, n, state):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for i in range(n):
            state.copy_(init)
            flush.fill_(1.0)
            torch.sum(flush, dim=0, out=sink)
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in zip(st, en))) / n

    steps = min(args.steps, 500)
    s_sur, s_pln = init.clone(), init.clone()
    nfb = torch.zeros(1, dtype=torch.int32, device=dev)
    sur = lambda: m.step(h, s_sur, wp, mdg.ACT_PID, N_SUB, 4.0, nfb, stream=stream)
    pln = lambda: h.step(s_pln, wp, mdg.ACT_PID, N_SUB, stream=stream)
    timed(sur, args.warmup, s_sur)
    timed(pln, args.warmup, s_pln)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms_sur = timed(sur, steps, s_sur)
    ms_pln = timed(pln, steps, s_pln)
    clk = clocks.stop()
    # the network kernel alone (tensor roofline)
    x = torch.empty((sw.n, mdg.MLP_IN_PAD), dtype=torch.bfloat16, device=dev)
    x.copy_(torch.randn_like(x, dtype=torch.float32).to(torch.bfloat16))
    y = torch.empty((sw.n, mdg.MLP_OUT_PAD), device=dev)
    ms_net = timed(lambda: m.forward(x, y, stream=stream), steps, s_sur)
    flops = 2.0 * sw.n * (64 * 256 + 2 * 256 * 256 + 256 * 32)
    # one-step accuracy from the initial swarm
    s_sur.copy_(init)
    s_pln.copy_(init)
    before = sg.state13(init).clone()
    sur()
    pln()
    torch.cuda.synchronize()
    xs, xp = sg.state13(s_sur), sg.state13(s_pln)
    true_d = xp - before
    zt = (true_d - out_mean) / out_std
    fb_env = ((xs - xp).abs().max(1).values.view(-1, 4) == 0).all(1).repeat_interleave(4)
    regular = (zt.abs() <= 8).all(1) & ~fb_env
    err = {}
    for name, sl in (("position", slice(0, 3)), ("quaternion", slice(3, 7)), ("velocity", slice(7, 10)),
                     ("body_rate", slice(10, 13))):
        e = float((xs[regular, sl] - xp[regular, sl]).pow(2).mean().sqrt())
        b = float(true_d[regular, sl].pow(2).mean().sqrt())
        err[name] = {"rms_error": e, "rms_change": b, "ratio_vs_no_network": e / b if b > 0 else None}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    ach = flops / (ms_net * 1e-3) / 1e12
    value = sw.n / (ms_sur * 1e-3)
    out = {
        "metric": "surrogate speedup at stated error: drone-control-steps/s of the surrogate step",
        "value": value, "unit": "drone-control-steps/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms_sur, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "surrogate: 65536 envs x 4 drones, PID waypoints, one control step; network "
                               "41-256-256-256-13 SiLU, bf16 weights/activations, FP32 accumulation, fused tcgen05 "
                               "kernel (two tiles in flight per block); out-of-distribution environments on the plain integrator",
                   "l2": "flushed between timed steps (512 MiB written, then read back)",
                   "training": {"transitions_generated": 16384 * 4 * 153, "transitions_kept": n_train,
                                "kept_fraction": kept, "epochs": 4, "batch": 8192, "seconds": train_s,
                                "loss_per_epoch": hist, "path": "tcgen05", "per_path": train_paths}},
        "plain_integrator": {"value": sw.n / (ms_pln * 1e-3), "ms_per_step": ms_pln},
        "speedup_vs_plain": ms_pln / ms_sur,
        "one_step_error_vs_plain": err, "regular_fraction": float(regular.float().mean()),
        "ood_env_fraction": int(nfb) / sw.n_envs,
        "gpu_launches": 5 * steps,
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_tflops"], "traffic": None, "peak_src": "measured (bf16 burst)",
                     "kernel": "mlp_umma_pair_kernel", "ms": ms_net, "algorithmic_flops_per_launch": flops},
        "clocks": clk,
    }
    print(json.dumps(out))


def run_surrogate_dense(args) -> None:
    """The learned surrogate on the dense swarm (1024 envs x 64 drones, all effects, the dense
    workload's RPM actions): trained on ~10.5M transitions of the plain integrator on fresh
    draws of the same workload (episodes of 40 control steps), with the integrator chosen by
    --integrator (Euler, or RK4 as the MuJoCo modes integrate), then one control step of the
    benchmark swarm with the surrogate against the plain step of the same integrator (both
    without observations, L2 flushed between steps). Metric: drone-control-steps/s of the
    surrogate step, with the plain step's figure, the one-step state error of the surrogate
    against the plain integrator on the regular regime, and the out-of-distribution fraction."""
    import torch
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import surrogate as sg
    from paper_2606_08039_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    c = library_constants(args)
    hover = c.hover_rpm()
    t0 = time.perf_counter()
    steps_gen, episode = 160, 40
    raw, delta = sg.generate_transitions(1024, steps_gen, seed=31, device=dev, workload="dense", constants=c,
                                         episode=episode)
    data = sg.Dataset(raw, delta)
    del raw, delta
    sw = wl.dense(5)
    m = mdg.MLP(sw.n, wl.mlp_init(3))
    data.attach(m)
    hist = sg.fit(m, data, epochs=4, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_train, kept, out_std, out_mean = len(data), data.kept_fraction, data.out_std, data.out_mean
    train_paths = training_step_ms(data)
    del data

    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    init = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
    act = torch.as_tensor(wl.rpm_actions(5, sw.n, 0, hover), device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def timed(fn, n, state):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for i in range(n):
            state.copy_(init)
            flush.fill_(1.0)
            torch.sum(flush, dim=0, out=sink)
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in zip(st, en))) / n

    steps = min(args.steps, 500)
    s_sur, s_pln = init.clone(), init.clone()
    nfb = torch.zeros(1, dtype=torch.int32, device=dev)
    sur = lambda: m.step(h, s_sur, act, mdg.ACT_RPM, N_SUB, 4.0, nfb, stream=stream)
    pln = lambda: h.step(s_pln, act, mdg.ACT_RPM, N_SUB, stream=stream)
    timed(sur, args.warmup, s_sur)
    timed(pln, args.warmup, s_pln)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms_sur = timed(sur, steps, s_sur)
    ms_pln = timed(pln, steps, s_pln)
    clk = clocks.stop()
    x = torch.empty((sw.n, mdg.MLP_IN_PAD), dtype=torch.bfloat16, device=dev)
    x.copy_(torch.randn_like(x, dtype=torch.float32).to(torch.bfloat16))
    y = torch.empty((sw.n, mdg.MLP_OUT_PAD), device=dev)
    ms_net = timed(lambda: m.forward(x, y, stream=stream), steps, s_sur)
    flops = 2.0 * sw.n * (64 * 256 + 2 * 256 * 256 + 256 * 32)
    # one-step accuracy from the benchmark swarm's initial state
    s_sur.copy_(init)
    s_pln.copy_(init)
    before = sg.state13(init).clone()
    sur()
    pln()
    torch.cuda.synchronize()
    xs, xp = sg.state13(s_sur), sg.state13(s_pln)
    true_d = xp - before
    zt = (true_d - out_mean) / out_std
    N = int(sw.drones_per_env[0])
    fb_env = ((xs - xp).abs().max(1).values.view(-1, N) == 0).all(1).repeat_interleave(N)
    regular = (zt.abs() <= 8).all(1) & ~fb_env
    err = {}
    for name, sl in (("position", slice(0, 3)), ("quaternion", slice(3, 7)), ("velocity", slice(7, 10)),
                     ("body_rate", slice(10, 13))):
        e = float((xs[regular, sl] - xp[regular, sl]).pow(2).mean().sqrt())
        b = float(true_d[regular, sl].pow(2).mean().sqrt())
        err[name] = {"rms_error": e, "rms_change": b, "ratio_vs_no_network": e / b if b > 0 else None}
    peaks = measured_peaks()
    ach = flops / (ms_net * 1e-3) / 1e12
    out = {
        "metric": "surrogate speedup at stated error: drone-control-steps/s of the surrogate step",
        "value": sw.n / (ms_sur * 1e-3), "unit": "drone-control-steps/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_sur, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"surrogate on the dense swarm: 1024 envs x 64 drones, all effects, RPM actions, one "
                               f"control step ({args.integrator} substeps in the plain step and the fallback); network "
                               "41-256-256-256-13 SiLU, bf16/FP32 accumulation, fused tcgen05 kernel",
                   "l2": "flushed between timed steps (512 MiB written, then read back)",
                   "training": {"transitions_generated": 1024 * 64 * steps_gen, "transitions_kept": n_train,
                                "kept_fraction": kept, "episode_steps": episode, "epochs": 4, "batch": 8192,
                                "seconds": train_s, "loss_per_epoch": hist, "path": "tcgen05",
                                "per_path": train_paths},
                   **model_config(args)},
        "plain_integrator": {"value": sw.n / (ms_pln * 1e-3), "ms_per_step": ms_pln,
                             "integrator": args.integrator},
        "speedup_vs_plain": ms_pln / ms_sur,
        "one_step_error_vs_plain": err, "regular_fraction": float(regular.float().mean()),
        "ood_env_fraction": int(nfb) / sw.n_envs,
        "gpu_launches": 5 * steps,
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_tflops"], "traffic": None, "peak_src": peaks["src"],
                     "kernel": "mlp_umma_pair_kernel", "ms": ms_net, "algorithmic_flops_per_launch": flops},
        "clocks": clk,
    }
    print(json.dumps(out))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mdg", choices=["mdg", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--episode-steps", type=int, default=EPISODE,
                    help="full_aero: control steps of the persistent-episode leg (the workload's episode: 1000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="full_aero",
                    choices=["full_aero", "uneven", "dense", "single", "surrogate", "surrogate_dense", "mlp",
                             "camera"],
                    help="full_aero (default, the headline line); the others measure the other swarms")
    ap.add_argument("--model", default="cf2x", choices=["cf2x", "cf2p", "race"])
    ap.add_argument("--integrator", default="euler", choices=["euler", "rk4"])
    ap.add_argument("--gnd-heights", default="com", choices=["com", "rotor"])
    ap.add_argument("--actions", default="pid", choices=sorted(ACTION_CHOICES),
                    help="full_aero: the action type of every environment, or mixed (all six types)")
    ap.add_argument("--controller", default="pid", choices=["pid", "dsl"])
    ap.add_argument("--envs", type=int, default=0, help="camera: environments rendered (default 16384, the swarm's size)")
    ap.add_argument("--randomize", action="store_true",
                    help="full_aero: domain randomization from the recommended ranges, motor lag, latency, wind")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in ("surrogate", "mlp", "camera") and not is_default_model(args):
        ap.error("--model/--integrator/--gnd-heights/--actions/--controller apply to the dynamics workloads only")
    if args.workload != "full_aero" and ((args.actions, args.controller) != ("pid", "pid") or args.randomize):
        ap.error("--actions/--controller/--randomize apply to the full_aero workload")
    if args.randomize and args.integrator == "rk4":
        ap.error("--randomize integrates with Euler substeps")
    if args.workload == "surrogate":
        run_surrogate(args)
        return
    if args.workload == "surrogate_dense":
        run_surrogate_dense(args)
        return
    if args.workload == "mlp":
        run_mlp(args)
        return
    if args.workload == "camera":
        run_camera(args)
        return
    if args.workload != "full_aero":
        run_other(args)
        return

    import torch
    import torch.distributed as dist
    import paper_2606_08039_gb300 as mdg
    from paper_2606_08039_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    # workload: N_SWARMS independent full-aero swarms per rank (swarm 0 is the rank's
    # replica), each with its own handle, state, waypoints and observation buffers
    c_lib = library_constants(args)
    act_type = mdg.ACT_MIXED if args.actions == "mixed" else ACTION_CHOICES[args.actions]

    class Swarm:
        def __init__(self, seed: int):
            sw = wl.full_aero(seed)
            self.sw = sw
            self.h = mdg.Handle(sw.drones_per_env, sw.flags, library_constants(args))
            self.init_state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=dev)
            self.state = self.init_state.clone()
            # the action of every drone: waypoints for the PID (the headline), else the chosen type
            self.types = action_types(args, sw.n_envs, seed)
            if args.actions == "pid":
                act_np = wl.waypoints(seed, sw.n)
            else:
                act_np = wl.typed_actions(sw.drones_per_env, self.types, seed, 0, c_lib.hover_rpm(),
                                          c_lib.mass * c_lib.g)
            if act_type == mdg.ACT_MIXED:
                self.h.set_action_types(self.types)
            self.setpoints = None
            if args.controller == "dsl":
                self.setpoints = self.h.new_setpoints(dev)
                self.h.set_setpoints(self.setpoints)
            self.dr_state = None
            if args.randomize:
                self.dr_state = self.h.new_randomization_state(DR_DEPTH, dev)
                table = torch.as_tensor(wl.dr_table(seed, sw.n_envs, depth=DR_DEPTH), device=dev)
                self.h.set_randomization(table, *self.dr_state, seed=DR_SEED)
            self.wp_host = torch.from_numpy(act_np).pin_memory()
            self.wp = self.wp_host.to(dev)
            self.kin, self.idx, self.rel = self.h.new_obs(dev)
            self.steps_done = 0

        def reset(self):
            self.state.copy_(self.init_state)
            if self.setpoints is not None:
                self.setpoints.fill_(float("nan"))
            if self.dr_state is not None:
                self.dr_state[0].fill_(float("nan"))
                self.dr_state[1].fill_(float("nan"))
                self.dr_state[2].zero_()
                self.dr_state[2][:, 3] = -1.0
            self.steps_done = 0

        def step(self, stream):
            self.h.step_obs(self.state, self.wp, act_type, N_SUB, self.kin, self.idx, self.rel, stream=stream)
            self.steps_done += 1

    swarms = [Swarm(replica_seed(rank) + SWARM_SEED_STRIDE * k) for k in range(N_SWARMS)]
    s0 = swarms[0]
    sw, h, types = s0.sw, s0.h, s0.types
    state, wp, wp_host, kin, idx, rel = s0.state, s0.wp, s0.wp_host, s0.kin, s0.idx, s0.rel
    reset = s0.reset
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_sink = torch.empty((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def flush_l2():
        flush.fill_(1.0)
        torch.sum(flush, dim=0, out=flush_sink)

    for i in range(args.warmup):
        swarms[i % N_SWARMS].step(stream)
    torch.cuda.synchronize()

    def capture(first_k):
        """One step of each of the first first_k swarms, in rotation, as one CUDA graph."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cap = torch.cuda.current_stream(dev)
            for sm in swarms[:first_k]:
                sm.h.step_obs(sm.state, sm.wp, act_type, N_SUB, sm.kin, sm.idx, sm.rel, stream=cap)
        return g

    graph = capture(N_SWARMS)  # 16 launches of the step kernel
    # regions hold a whole number of rotations except the last one, which ends with one step
    # of each of the first steps % 16 swarms: that tail is a graph too
    tail_graph = capture(args.steps % N_SWARMS) if args.steps % N_SWARMS else None
    for sm in swarms:
        sm.reset()
        sm.h.status()
    torch.cuda.synchronize()

    # Timed region: K control steps back to back, swarm after swarm (inputs larger than L2:
    # each swarm's state, waypoints and observations are touched again only after the 15
    # other swarms' 299 MB), events around the whole region. Every launch of the region is in
    # a CUDA graph (the 16-swarm rotation, then one graph of the first steps % 16 swarms), and
    # a bounded device sleep before the start event keeps the GPU busy while the host submits
    # them, so the events see back-to-back device time at any step count. Every swarm is reset
    # to its initial state outside the region; a region holds at most one episode per swarm.
    seg_max = N_SWARMS * EPISODE
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region
    total_ms = 0.0
    wall = 0.0
    windows = []
    remaining = args.steps
    while remaining:
        n_seg = min(remaining, seg_max)
        for sm in swarms:
            if sm.steps_done:
                sm.reset()
        flush_l2()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        torch.cuda._sleep(HEAD_START_CYCLES)
        ev0.record(stream)
        for _ in range(n_seg // N_SWARMS):
            graph.replay()
        if n_seg % N_SWARMS:
            tail_graph.replay()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        windows.append((wall0, time.perf_counter()))
        wall += windows[-1][1] - wall0
        total_ms += ev0.elapsed_time(ev1)
        for k, sm in enumerate(swarms):
            sm.steps_done += n_seg // N_SWARMS + (1 if k < n_seg % N_SWARMS else 0)
        remaining -= n_seg
    clk = clocks.stop(windows)
    nonfinite = False
    for sm in swarms:
        rc, bits, first = sm.h.status()
        nonfinite = nonfinite or bool(bits & mdg.STATUS_NONFINITE)
    nonfinite_frac = nonfinite_fraction([sm.state for sm in swarms])

    # The same step isolated: swarm 0 alone, the L2 flushed before every step and every
    # step bracketed by its own events (launch and timestamp latency included per step).
    n_iso = min(args.steps, ISOLATED_STEPS)
    reset()
    iso_starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_iso)]
    iso_ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_iso)]
    for i in range(n_iso):
        flush_l2()
        iso_starts[i].record(stream)
        s0.step(stream)
        iso_ends[i].record(stream)
    torch.cuda.synchronize()
    iso_ms = float(sum(a.elapsed_time(b) for a, b in zip(iso_starts, iso_ends)))
    h.status()

    # end to end through the public API with host buffers
    kin_h = torch.empty(kin.shape, dtype=kin.dtype).pin_memory()
    idx_h = torch.empty(idx.shape, dtype=idx.dtype).pin_memory()
    rel_h = torch.empty(rel.shape, dtype=rel.dtype).pin_memory()
    e_starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
    e_ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
    reset()
    # the step kernel reads the waypoints from, and writes the observations to, the pinned
    # host buffers itself (mdg_step_obs_host): the transfers overlap its arithmetic. Under
    # randomization (whose observation noise and delay the host-buffer path does not take)
    # the waypoints are copied in and the observations copied out around mdg_step_obs.
    for i in range(args.e2e_steps):
        flush_l2()
        e_starts[i].record(stream)
        if args.randomize:
            wp.copy_(wp_host, non_blocking=True)
            h.step_obs(state, wp, act_type, N_SUB, kin, idx, rel, stream=stream)
            kin_h.copy_(kin, non_blocking=True)
            idx_h.copy_(idx, non_blocking=True)
            rel_h.copy_(rel, non_blocking=True)
        else:
            h.step_obs_host(state, wp_host, act_type, N_SUB, kin_h, idx_h, rel_h, stream=stream)
        e_ends[i].record(stream)
        e_ends[i].synchronize()
    e2e_ms = float(sum(s.elapsed_time(e) for s, e in zip(e_starts, e_ends)))
    h2d = wp_host.numel() * 4
    d2h = kin_h.numel() * 4 + idx_h.numel() * 4 + rel_h.numel() * 4

    # The workload's 1000-control-step episode as one persistent rollout (mdg_rollout): the
    # state stays in registers across steps, the PID waypoints are fixed for the episode and
    # the observations of every step are written ([K][n] buffers, 12.6 GB). L2 flushed
    # between episodes.
    episode = args.episode_steps
    ep_kin = torch.empty((episode,) + tuple(kin.shape), dtype=kin.dtype, device=dev)
    ep_idx = torch.empty((episode,) + tuple(idx.shape), dtype=idx.dtype, device=dev)
    ep_rel = torch.empty((episode,) + tuple(rel.shape), dtype=rel.dtype, device=dev)
    ep_starts = [torch.cuda.Event(enable_timing=True) for _ in range(EPISODE_REPS)]
    ep_ends = [torch.cuda.Event(enable_timing=True) for _ in range(EPISODE_REPS)]
    for i in range(1 + EPISODE_REPS):
        reset()
        flush_l2()
        if i:
            ep_starts[i - 1].record(stream)
        h.rollout(state, wp, act_type, N_SUB, episode, mdg.OBS_EVERY_STEP, ep_kin, ep_idx, ep_rel, stream=stream)
        if i:
            ep_ends[i - 1].record(stream)
    torch.cuda.synchronize()
    ep_ms = float(sum(a.elapsed_time(b) for a, b in zip(ep_starts, ep_ends)))
    del ep_kin, ep_idx, ep_rel

    total_ms, e2e_ms, ep_ms, iso_ms = combine_over_ranks([total_ms, e2e_ms, ep_ms, iso_ms], world, device=dev)
    value = throughput(sw.n * N_SUB, world, args.steps, total_ms)
    e2e_value = throughput(sw.n * N_SUB, world, args.e2e_steps, e2e_ms)
    iso_value = throughput(sw.n * N_SUB, world, n_iso, iso_ms)

    if rank == 0:
        peaks = measured_peaks()
        avg_s = total_ms / args.steps * 1e-3
        bytes_launch = algorithmic_bytes(sw, types, act_type, args.controller == "dsl",
                                         DR_DEPTH if args.randomize else 0)
        loops_mask = np.isin(types, (1, 5, 6))  # PID, VEL, ATTITUDE run the controller loops
        flops_launch = algorithmic_flops(sw, 1, N_SUB, 1, loops_mask, rk4=args.integrator == "rk4")
        roofline = binding_roofline(bytes_launch, flops_launch, avg_s, peaks)
        # the ncu capture is of the default configuration's kernel at this source
        roofline["traffic"] = (NCU_TRAFFIC["bytes"] if NCU_TRAFFIC["kernel_sha"] == kernel_sha()
                               and is_default_model(args) else None)
        roofline["kernel"] = "step_kernel<obs>"
        roofline["kernel_sha"] = kernel_sha()
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "full_aero: 16384 envs x 4 Crazyflie 2.x, ground effect + drag + downwash, "
                                   "PID waypoints, 240 Hz physics / 48 Hz control (5 substeps), KIN + 4-NN obs; "
                                   "one step = one control step (one fused kernel launch)",
                       "n_drones_per_gpu": sw.n, "n_substeps": N_SUB, "block_size": h.block_size,
                       "l2": f"inputs larger than L2: {N_SWARMS} independent swarms of this size stepped in "
                             f"rotation, each swarm's {SWARM_BYTES / 2**20:.0f} MiB of state, waypoints and "
                             f"observations touched again after the other swarms' "
                             f"{(N_SWARMS - 1) * SWARM_BYTES / 2**20:.0f} MiB; no flush inside the timed region",
                       "timing": f"CUDA graph of {N_SWARMS} step launches (one per swarm) replayed back to back, "
                                 f"then a graph of the first steps % {N_SWARMS} swarms; a bounded device sleep "
                                 "before the start event (host submission overlapped); events around the whole "
                                 "timed region",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": args.e2e_steps,
                    "path": ("mdg_step_obs with the waypoints copied in from and the observations copied out to "
                             "pinned host memory around it, synchronised on every step" if args.randomize else
                             "mdg_step_obs_host: waypoints read and observations written in pinned host memory "
                             "by the step kernel, synchronised on every step")},
            "gpu_launches": args.steps,
            "roofline": roofline,
            "clocks": clk,
            "wall_s_timed_region": wall,
            "nonfinite_during_timing": nonfinite,
            "nonfinite_fraction_after_timing": nonfinite_frac,
            "episode": episode_line(sw.n, world, ep_ms, peaks, flops_launch, episode),
            "isolated_step": {
                "what": "swarm 0 alone, L2 flushed (512 MiB written, then read back) before every step, every "
                        "step bracketed by its own events: one launch's latency and timestamps included per step",
                "value": iso_value, "unit": UNIT, "ms_per_step": iso_ms / n_iso, "steps": n_iso,
                "roofline": binding_roofline(bytes_launch, flops_launch, iso_ms / n_iso * 1e-3, peaks)},
        }
        out["config"].update(model_config(args))
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
