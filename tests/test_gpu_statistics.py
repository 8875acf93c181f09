"""Long rollouts of the chaotic workloads compared statistically.

Downwash at near-coincident heights (Eq. downwash: force ~ 1/dz^2) amplifies a rounding
difference of one float32 ulp into a visibly different trajectory within a few control
steps, so beyond a short horizon the GPU's FP32 trajectory and the FP64 oracle's cannot be
compared drone by drone (the per-step restart protocol of the other parity tests covers
that). Here both run the same swarm independently from the same initial state for many
control steps, with Euler or RK4 substeps, and their ensembles are compared at regular
snapshots (helpers.ensemble_check:
KS tests of height, speed and body-rate magnitude with a Bonferroni level, means within 3
standard errors, non-finite fractions within 3 binomial standard errors). Everything is
seeded, so each comparison is one fixed outcome, not a random draw.

What the comparison can see is pinned on the CPU in test_statistics_power below: it passes
for the oracle against itself with every height moved by one float32 ulp, and fails for
the oracle with one of a few plausible mistakes (MUTATIONS; under RK4 on full aero also
Euler substeps in its place). Smaller errors (downwash off
by 20%, gravity by 1%) stay inside its statistical resolution; the per-substep parity
tests are the ones that see those.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from paper_2606_08039_gb300 import workloads as wl
from helpers import ensemble_check, oracle_arrays, oracle_snapshots

HOVER = oracle.hover_rpm(oracle.cf2x())
CASES = {"full_aero": (200, 10), "dense": (40, 4)}  # control steps, snapshot interval
INTEGRATORS = {"euler": (mdg.INTEGRATOR_EULER, oracle.EULER), "rk4": (mdg.INTEGRATOR_RK4, oracle.RK4)}


def _params(integrator):
    P = oracle.cf2x()
    P.integrator = INTEGRATORS[integrator][1]
    return P


def _swarm(recipe):
    K = CASES[recipe][0]
    if recipe == "full_aero":
        sw = wl.full_aero(61, n_envs=1024)
        return sw, mdg.ACT_PID, np.broadcast_to(wl.waypoints(61, sw.n), (K, sw.n, 4)).astype(np.float32)
    sw = wl.dense(62, n_envs=32)
    return sw, mdg.ACT_RPM, np.stack([wl.rpm_actions(62, sw.n, k, HOVER) for k in range(K)])


@pytest.mark.gpu
@pytest.mark.parametrize("integrator", sorted(INTEGRATORS))
@pytest.mark.parametrize("recipe", sorted(CASES))
def test_long_rollout_statistics(cuda, recipe, integrator):
    pytest.importorskip("scipy.stats")
    K, every = CASES[recipe]
    sw, act_type, actions = _swarm(recipe)
    c = mdg.Constants.cf2x()
    c.integrator = INTEGRATORS[integrator][0]
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    gpu = []
    for k0 in range(0, K, every):
        if recipe == "full_aero":  # one launch per control step
            wp = torch.as_tensor(np.ascontiguousarray(actions[k0]), device=cuda)
            for _ in range(every):
                h.step(state, wp, act_type, 5)
        else:  # persistent rollouts of `every` steps
            h.rollout(state, torch.as_tensor(np.ascontiguousarray(actions[k0:k0 + every]), device=cuda), act_type, 5,
                      every)
        torch.cuda.synchronize()
        gpu.append(oracle_arrays(state)[0])
    ref = oracle_snapshots(_params(integrator), sw, act_type, actions, every)
    ok, why = ensemble_check(gpu, ref)
    assert ok, f"{recipe} {integrator}: {why}"
    assert h.status()[0] in (mdg.OK, mdg.ERR_NONFINITE)


# mutations each comparison must reject: (field, factor); blade drag removal sets c_z too
MUTATIONS = {"full_aero": (("c_xy", 0.0), ("c_gnd", 0.0)), "dense": (("dw_c1", 0.5), ("kf", 1.05))}


@pytest.mark.parametrize("integrator", sorted(INTEGRATORS))
@pytest.mark.parametrize("recipe", sorted(CASES))
def test_statistics_power(recipe, integrator):
    """CPU: the ensemble comparison accepts a one-ulp perturbation of every height (a
    different but equally valid chaotic trajectory) and rejects the same swarm simulated
    with a plausible mistake: full aero without blade drag or without ground effect, the
    dense swarm with half the downwash or a 5% larger thrust coefficient. (Ground effect is
    invisible in the dense lattice, whose lowest layer flies at 0.5 m.) Under RK4 the full-aero
    comparison also rejects Euler substeps in its place; on the dense lattice the two
    integrators' ensembles are not distinguishable."""
    pytest.importorskip("scipy.stats")
    K, every = CASES[recipe]
    sw, act_type, actions = _swarm(recipe)
    P = _params(integrator)
    ref = oracle_snapshots(P, sw, act_type, actions, every)
    x0 = np.concatenate([sw.p, sw.q, sw.v, sw.w], axis=1).astype(np.float64)
    x0[:, 2] = np.nextafter(sw.p[:, 2].astype(np.float32), np.float32(np.inf))
    ok, why = ensemble_check(oracle_snapshots(P, sw, act_type, actions, every, x0=x0), ref)
    assert ok, why
    mutations = MUTATIONS[recipe] + ((("integrator", None),) if (recipe, integrator) == ("full_aero", "rk4") else ())
    for field, factor in mutations:
        Pm = _params(integrator)
        if field == "integrator":
            Pm.integrator = oracle.EULER
            ok, _ = ensemble_check(oracle_snapshots(Pm, sw, act_type, actions, every), ref)
            assert not ok, f"{recipe}: Euler in place of RK4 not detected"
            continue
        setattr(Pm, field, getattr(Pm, field) * factor)
        if field == "c_xy":
            Pm.c_z = 0.0
        ok, _ = ensemble_check(oracle_snapshots(Pm, sw, act_type, actions, every), ref)
        assert not ok, f"{recipe}: {field} x {factor} not detected"
