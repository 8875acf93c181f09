"""Training and evaluation of the learned surrogate on transitions of the simulator itself.

The network (MLP, C ABI mdg_mlp_*) learns the 13-d state change of one control step from
the 41 inputs the library builds (state, RPMs, 4 nearest neighbours' relative state).
Transitions come from the GPU simulator (mdg_transition: the inputs, one plain control step,
the state change), on the full-aero swarm with PID RPMs towards random waypoints, each motor
perturbed by a factor U[1 - perturb, 1 + perturb] drawn by the input generator, or on the
dense swarm with its RPM actions. The standardisation of the training set (trim, mean and
standard deviation, out-of-distribution box: mdg_mlp_fit_normalization) and every
computation of the network (forward, backward, Adam) run in the library's kernels; this
module only moves tensors: batching, shuffling and the learning-rate schedule.
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
    applied = torch.empty((sw.n, 4), dtype=torch.float32, device=device)
    idx = np.arange(sw.n, dtype=np.uint64)[:, None]
    comp = np.arange(4, dtype=np.uint64)[None, :]
    for k in range(steps):
        if episode and k and k % episode == 0:
            fresh = make(seed + 7919 * (k // episode), n_envs)
            state.copy_(mdg.pack_state(fresh.p, fresh.q, fresh.v, fresh.w, device=device))
        if workload == "full_aero":
            h.pid(state, wp, rpm)
            scale = torch.as_tensor(wl.uniform_range(1.0 - perturb, 1.0 + perturb, seed, wl.S_ACT, 1000 + k, idx, comp),
                                    device=device)
        else:
            rpm.copy_(torch.as_tensor(wl.rpm_actions(seed, sw.n, k, hover), device=device))
            scale = None
        h.transition(state, rpm, applied, raw[k], delta[k], rpm_scale=scale, n_substeps=n_substeps)
    return raw.reshape(-1, mdg.MLP_IN), delta.reshape(-1, mdg.MLP_OUT)


class Dataset:
    """Standardised training set (bf16 inputs [N, 64], FP32 targets [N, 32]) of a set of
    transitions and its statistics (mdg_mlp_fit_normalization, held by a small network that
    carries the normalisation: attach() gives it to the network that trains)."""

    def __init__(self, raw, delta, ood_z: float = 4.0, target_clip: float = 8.0):
        torch = _torch()
        import paper_2606_08039_gb300 as mdg
        N = raw.shape[0]
        self._holder = mdg.MLP(128)
        x = torch.empty((N, mdg.MLP_IN_PAD), dtype=torch.bfloat16, device=raw.device)
        t = torch.empty((N, mdg.MLP_OUT_PAD), dtype=torch.float32, device=raw.device)
        n_fin, n = self._holder.fit_normalization(raw, delta, x, t, ood_z=ood_z, target_clip=target_clip)
        self.x, self.t = x[:n], t[:n]
        self.kept_fraction = n / max(1, n_fin)
        self.ood_z = ood_z
        (in_mean, in_std, out_mean, out_std, in_lo, in_hi) = self._holder.normalization()
        dev = raw.device
        self.in_mean, self.in_std = torch.as_tensor(in_mean, device=dev), torch.as_tensor(in_std, device=dev)
        self.out_mean, self.out_std = torch.as_tensor(out_mean, device=dev), torch.as_tensor(out_std, device=dev)
        self.in_lo, self.in_hi = torch.as_tensor(in_lo, device=dev), torch.as_tensor(in_hi, device=dev)

    def stats(self):
        return self._holder.normalization()

    def attach(self, mlp):
        """Give the network this set's normalisation."""
        mlp.set_normalization(*self.stats())

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
