"""Training and evaluation of the learned surrogate on transitions of the simulator itself.

The network (MLP, C ABI mdg_mlp_*) learns the 13-d state change of one control step from
the 41 inputs mdg_features builds (state, RPMs, 4 nearest neighbours' relative state).
Transitions come from the GPU simulator on the full-aero swarm: PID RPMs towards random
waypoints, each motor perturbed by U[1 - perturb, 1 + perturb] for diversity, then one
plain control step. Every computation of the network (forward, backward, Adam, input
standardisation) runs in the library's kernels; this module only moves tensors:
shuffling, batching and the normalisation statistics.

Normalisation: transitions are trimmed per dimension to the central 99% of inputs and
targets (plus a 10% margin of that range) — the excluded tail is dominated by the chaotic
near-coincident heights of the downwash law — and the mean and standard deviation of the
kept set standardise inputs and targets (scale 1 where a feature is constant). The
surrogate step sends an environment to the plain integrator when a drone's standardised
input leaves +-ood_z or its raw input leaves the kept set's box (plus 10%).
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as wl


def _torch():
    import torch
    return torch


def state13(state):
    """[6, n, 4] state planes -> [n, 13] = p, q, v, omega (torch, same device)."""
    torch = _torch()
    s = state
    return torch.cat([s[0, :, 0:3], s[0, :, 3:4], s[1, :, 0:3], s[1, :, 3:4], s[2, :, 0:2], s[2, :, 2:4],
                      s[3, :, 0:1]], dim=1)


def generate_transitions(n_envs: int, steps: int, seed: int, device, perturb: float = 0.1, n_substeps: int = 5,
                         workload: str = "full_aero", constants=None, episode: int = 0):
    """Transitions of a swarm under the library's plain integrator (the handle's constants:
    Euler or RK4 substeps): (raw inputs [steps * n, 41], state change [steps * n, 13]).
    full_aero: PID RPMs towards the workload's waypoints, each motor times U[1 - perturb,
    1 + perturb]; dense: the dense workload's RPM actions (hover times U[0.9, 1.1] per motor).
    episode > 0: the swarm restarts from a fresh draw of its workload every `episode` steps."""
    torch = _torch()
    import paper_2606_08039_gb300 as mdg
    make = {"full_aero": wl.full_aero, "dense": wl.dense}[workload]
    sw = make(seed, n_envs)
    h = mdg.Handle(sw.drones_per_env, sw.flags, constants)
    hover = (constants or mdg.Constants.cf2x()).hover_rpm()
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=device)
    wp = torch.as_tensor(wl.waypoints(seed, sw.n), device=device)
    raw = torch.empty((steps, sw.n, mdg.MLP_IN), dtype=torch.float32, device=device)
    delta = torch.empty((steps, sw.n, mdg.MLP_OUT), dtype=torch.float32, device=device)
    rpm = torch.empty((sw.n, 4), dtype=torch.float32, device=device)
    idx = np.arange(sw.n, dtype=np.uint64)[:, None]
    comp = np.arange(4, dtype=np.uint64)[None, :]
    for k in range(steps):
        if episode and k and k % episode == 0:
            fresh = make(seed + 7919 * (k // episode), n_envs)
            state.copy_(mdg.pack_state(fresh.p, fresh.q, fresh.v, fresh.w, device=device))
        if workload == "full_aero":
            h.pid(state, wp, rpm)
            noise = wl.uniform_range(1.0 - perturb, 1.0 + perturb, seed, wl.S_ACT, 1000 + k, idx, comp)
            rpm.mul_(torch.as_tensor(noise, device=device))
        else:
            rpm.copy_(torch.as_tensor(wl.rpm_actions(seed, sw.n, k, hover), device=device))
        h.features(state, rpm, raw[k])
        before = state13(state).clone()
        h.step(state, rpm, mdg.ACT_RPM, n_substeps)
        delta[k] = state13(state) - before
    return raw.reshape(-1, mdg.MLP_IN), delta.reshape(-1, mdg.MLP_OUT)


def _trim_box(a, frac: float = 0.005, margin: float = 0.1):
    """Per-column [q(frac) - margin r, q(1 - frac) + margin r], r the quantile range, on an
    evenly strided sample of at most 262144 rows."""
    torch = _torch()
    stride = max(1, a.shape[0] // 262144)
    q = torch.quantile(a[::stride].float(), torch.tensor([frac, 1.0 - frac], device=a.device), dim=0)
    r = q[1] - q[0]
    return q[0] - margin * r, q[1] + margin * r


def _mean_std(a):
    torch = _torch()
    mean = a.double().mean(0)
    std = a.double().std(0)
    std = torch.where(std > 1e-6 * torch.clamp(mean.abs(), min=1.0), std, torch.ones_like(std))
    return mean.float(), std.float()


class Dataset:
    """Standardised training set (bf16 inputs [N, 64], FP32 targets [N, 32]) and its statistics."""

    def __init__(self, raw, delta, ood_z: float = 4.0, target_clip: float = 8.0):
        torch = _torch()
        import paper_2606_08039_gb300 as mdg
        finite = torch.isfinite(raw).all(1) & torch.isfinite(delta).all(1)
        raw, delta = raw[finite], delta[finite]
        ilo, ihi = _trim_box(raw)
        olo, ohi = _trim_box(delta)
        keep = ((raw >= ilo) & (raw <= ihi)).all(1) & ((delta >= olo) & (delta <= ohi)).all(1)
        raw, delta = raw[keep], delta[keep]
        self.in_mean, self.in_std = _mean_std(raw)
        self.out_mean, self.out_std = _mean_std(delta)
        zin = (raw - self.in_mean) / self.in_std
        keep2 = (zin.abs() <= ood_z).all(1) & (((delta - self.out_mean) / self.out_std).abs() <= target_clip).all(1)
        self.kept_fraction = float(keep.float().mean()) * float(keep2.float().mean())
        raw = raw[keep2]
        zout = ((delta - self.out_mean) / self.out_std)[keep2]
        lo, hi = raw.min(0).values, raw.max(0).values
        pad = 0.1 * (hi - lo) + 1e-6
        self.in_lo, self.in_hi = lo - pad, hi + pad
        self.ood_z = ood_z
        n = raw.shape[0] // 128 * 128
        self.raw = raw[:n]
        self.t = torch.zeros((n, mdg.MLP_OUT_PAD), dtype=torch.float32, device=raw.device)
        self.t[:, :mdg.MLP_OUT] = zout[:n]
        self.x = torch.empty((n, mdg.MLP_IN_PAD), dtype=torch.bfloat16, device=raw.device)

    def stats(self):
        return [t.detach().cpu().numpy().astype(np.float32) for t in
                (self.in_mean, self.in_std, self.out_mean, self.out_std, self.in_lo, self.in_hi)]

    def attach(self, mlp):
        """Give the network these statistics and standardise the inputs with its kernel."""
        mlp.set_normalization(*self.stats())
        mlp.standardize(self.raw, self.x)

    def __len__(self):
        return self.x.shape[0]


def fit(mlp, data: Dataset, epochs: int = 8, batch: int = 8192, lr: float = 2e-3, seed: int = 0):
    """Adam on the MSE of standardised targets, cosine-decayed learning rate, reshuffled
    every epoch. Returns the mean training loss of each epoch."""
    torch = _torch()
    gen = torch.Generator(device=data.x.device)
    gen.manual_seed(seed)
    n_b = len(data) // batch
    total = epochs * n_b
    loss = torch.zeros(1, dtype=torch.float32, device=data.x.device)
    hist = []
    it = 0
    for _ in range(epochs):
        perm = torch.randperm(len(data), generator=gen, device=data.x.device)
        acc = torch.zeros(1, dtype=torch.float64, device=data.x.device)
        for b in range(n_b):
            idx = perm[b * batch:(b + 1) * batch]
            xb = data.x.index_select(0, idx)
            tb = data.t.index_select(0, idx)
            mlp.grad(xb, tb, loss)
            acc += loss.double()
            mlp.adam(lr * 0.5 * (1.0 + math.cos(math.pi * it / max(1, total))) + 1e-5)
            it += 1
        hist.append(float(acc) / max(1, n_b))
    return hist
