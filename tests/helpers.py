"""Shared helpers of the parity tests: layout conversion between the library's state
planes and the oracle's [n, 13] arrays, and the tolerance checks.

Tolerances (stated once, used everywhere):
  per substep, restarted from the GPU's own float32 state:
      position, velocity  |gpu - ref| <= 1e-5 * max(|ref|, 1)   (m, m/s)
      body rate           |gpu - ref| <= 1e-4 * max(|ref|, 1)   (rad/s)
      quaternion          |gpu - ref| <= 2e-6
  The floor of 1 unit keeps the test relative for large values and absolute near zero,
  where a sum of terms that cancel has no meaningful relative error.
  neighbour lists (several are correct: float32 can order two distances that FP64 tells
  apart either way when they differ by less than its rounding):
      the same number of neighbours as the FP64 oracle, distinct other drones of the
      environment, and slot by slot a squared FP64 distance within KNN_RTOL of the
      oracle's in that slot
"""
import numpy as np

import oracle
import paper_2606_08039_gb300 as mdg

RTOL_PV = 1e-5
RTOL_W = 1e-4
ATOL_Q = 2e-6
# A float32 squared distance ((dx dx + dy dy) + dz dz) from float32 positions carries a
# relative error below 5 units of 2^-24 (3.0e-7): one rounding for each difference, product
# and sum. Two such values can be ordered wrongly only if their FP64 values differ by less than
# twice that, and the k-th smallest of the rounded values is then within the same relative
# bound of the oracle's k-th smallest: 1e-6 covers both with a margin.
KNN_RTOL = 1e-6


def oracle_arrays(state_tensor):
    """Library state [6, n, 4] -> (x [n,13], integ [n,6], a_prev [n,4]) in float64."""
    s = mdg.unpack_state(state_tensor)
    x = np.concatenate([s["p"], s["q"], s["v"], s["w"]], axis=1).astype(np.float64)
    integ = np.concatenate([s["ip"], s["ia"]], axis=1).astype(np.float64)
    return x, integ, s["a_prev"].astype(np.float64)


def swarm_state(swarm, device):
    return mdg.pack_state(swarm.p, swarm.q, swarm.v, swarm.w, device=device)


def excess(gpu, ref, rtol, floor=1.0):
    """Largest |gpu - ref| / (rtol * max(|ref|, floor)); <= 1 passes."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(gpu - ref) / (rtol * np.maximum(np.abs(ref), floor)), initial=0.0))


def assert_state_close(xg, xo, scale=1.0, what=""):
    """Compare [n,13] states with the per-substep tolerances times `scale`."""
    e_p = excess(xg[:, 0:3], xo[:, 0:3], RTOL_PV * scale)
    e_v = excess(xg[:, 7:10], xo[:, 7:10], RTOL_PV * scale)
    e_w = excess(xg[:, 10:13], xo[:, 10:13], RTOL_W * scale)
    e_q = float(np.max(np.abs(xg[:, 3:7] - xo[:, 3:7]), initial=0.0)) / (ATOL_Q * scale)
    worst = max(e_p, e_v, e_w, e_q)
    assert worst <= 1.0, f"{what}: tolerance exceeded (p {e_p:.3g}, v {e_v:.3g}, w {e_w:.3g}, q {e_q:.3g})"
    return worst


def oracle_step(P, swarm_or_layout, x, integ, a_prev, action, act_types, n_sub, obs=False):
    """One control step of the oracle on the given batch layout."""
    dpe, flags = swarm_or_layout
    env_off = np.concatenate([[0], np.cumsum(dpe)]).astype(np.int32)
    return oracle.control_steps(P, env_off, np.asarray(flags, np.int32), np.asarray(act_types, np.int32),
                                x, integ, a_prev, np.asarray(action, np.float64)[None], n_sub, obs=obs)


def spread_heights(sw, dz=0.3, z0=0.5):
    """The swarm with the drones of every environment at heights z0, z0 + dz, ... (in drone
    order; x, y and everything else unchanged)."""
    off = np.concatenate([[0], np.cumsum(sw.drones_per_env)])
    p = sw.p.copy()
    for e in range(sw.n_envs):
        p[off[e]:off[e + 1], 2] = z0 + dz * np.arange(off[e + 1] - off[e])
    sw.p = p.astype(np.float32)
    return sw


def subset_layout(dpe, envs):
    """Drone indices and layout of a subset of environments."""
    env_off = np.concatenate([[0], np.cumsum(dpe)])
    idx = np.concatenate([np.arange(env_off[e], env_off[e + 1]) for e in envs]) if len(envs) else np.zeros(0, int)
    return idx, np.asarray(dpe)[envs]


def tolerance_response(P, layout, x, integ, a_prev, action, act_types, n_sub, seed=0):
    """The oracle's own response over the horizon to an error of exactly the per-substep
    tolerance in the initial state (position and velocity by RTOL_PV * max(|.|, 1), body rate
    by RTOL_W * max(|.|, 1), quaternion by ATOL_Q, random signs). Chaotic downwash at small
    height differences amplifies any such error; this measures by how much. Returns |dx| [n,13]."""
    rng = np.random.default_rng(seed)
    x2 = x.copy()
    sgn = rng.choice([-1.0, 1.0], size=x.shape)
    for sl, tol in ((slice(0, 3), RTOL_PV), (slice(7, 10), RTOL_PV), (slice(10, 13), RTOL_W)):
        x2[:, sl] = x[:, sl] + sgn[:, sl] * tol * np.maximum(np.abs(x[:, sl]), 1.0)
    q = x[:, 3:7] + sgn[:, 3:7] * ATOL_Q
    x2[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    a = oracle_step(P, layout, x, integ, a_prev, action, act_types, n_sub)[0]
    b = oracle_step(P, layout, x2, integ, a_prev, action, act_types, n_sub)[0]
    return np.abs(a - b)


# Share of drones whose horizon bound is set by the dynamics' amplification rather than by the
# tolerance in a component other than height and vertical velocity: the downwash's 1/dz^2 law
# at near-equal heights amplifies an error mostly along z (measured with the oracle alone:
# full aero 0.25% of drones, dense 7.3%; the single drone none).
LOOSE_FACTOR = 10.0
VERTICAL = (2, 9)


def loose_share(xo, response):
    """Share of drones with any component other than z and v_z whose response exceeds
    LOOSE_FACTOR times its per-substep tolerance (there the horizon bound is wide)."""
    tol = np.zeros(13)
    tol[0:3] = tol[7:10] = RTOL_PV
    tol[10:13] = RTOL_W
    base = tol[None, :] * np.maximum(np.abs(xo), 1.0)
    base[:, 3:7] = ATOL_Q
    r = np.delete(response / base, VERTICAL, axis=1)
    return float((r > LOOSE_FACTOR).any(axis=1).mean()) if len(r) else 0.0


def assert_horizon_close(xg, xo, response, n_sub, what="", max_loose=None):
    """Short-horizon comparison over n_sub substeps: per component,
    |gpu - ref| <= n_sub * (tol * max(|ref|, 1) + response), where `response` is
    tolerance_response(): each of the n_sub substeps may add an error up to the per-substep
    tolerance, and the dynamics propagate it at most like an error of that size at the start
    (linear propagation of the per-substep bound). With max_loose, also that on all but that
    share of the drones every component other than z and v_z is held to
    n_sub * (1 + LOOSE_FACTOR) * tolerance (loose_share), so that the bound is not wide
    everywhere."""
    tol = np.zeros(13)
    tol[0:3] = tol[7:10] = RTOL_PV
    tol[10:13] = RTOL_W
    base = tol[None, :] * np.maximum(np.abs(xo), 1.0)
    base[:, 3:7] = ATOL_Q
    if max_loose is not None:
        share = loose_share(xo, response)
        assert share <= max_loose, f"{what}: horizon bound wide on {share:.1%} of the drones"
    bound = n_sub * (base + response)
    err = np.abs(xg - xo)
    ratio = err / bound
    worst = float(np.max(ratio, initial=0.0))
    if worst > 1.0:
        i, k = np.unravel_index(np.argmax(ratio), ratio.shape)
        raise AssertionError(f"{what}: drone {i} component {k}: gpu {xg[i, k]!r} oracle {xo[i, k]!r} "
                             f"bound {bound[i, k]:.3g} (ratio {worst:.3g})")
    return worst


def assert_knn_valid(x_env, j, base, idx_row, what=""):
    """The GPU's neighbour list idx_row (global indices, -1 padding) of drone j of one
    environment (x_env [N, 13] float64 of the float32 state the GPU observed; base = global
    index of the environment's first drone), checked against the FP64 oracle's selection
    (oracle.knn): as many entries as the oracle lists, -1 after them, distinct drones of the
    environment other than j, and in every slot k a squared FP64 distance within KNN_RTOL
    (relative) of the oracle's k-th. Returns (features [24] of the GPU's chosen drones in
    FP64: [p_i - p_j, v_i - v_j] per slot, zeros for padding; True if the list is the
    oracle's own)."""
    x_env = np.asarray(x_env, np.float64)
    got = np.asarray(idx_row).astype(np.int64)
    i_ref, r_ref = oracle.knn(x_env, j, base)
    n_ref = int((i_ref >= 0).sum())
    assert np.all(got[:n_ref] >= 0) and np.all(got[n_ref:] == -1), f"{what}: list {got}, oracle {i_ref}"
    loc = got[:n_ref] - base
    assert np.all((loc >= 0) & (loc < x_env.shape[0]) & (loc != j)), f"{what}: list {got} outside the environment"
    assert len(set(loc.tolist())) == n_ref, f"{what}: repeated neighbour in {got}"
    d2 = np.sum((x_env[:, 0:3] - x_env[j, 0:3]) ** 2, axis=1)
    dg, dr = d2[loc], d2[i_ref[:n_ref] - base]
    bad = np.abs(dg - dr) > KNN_RTOL * np.maximum(dg, dr)
    assert not bad.any(), f"{what}: list {got} (squared distances {dg}), oracle {i_ref} ({dr})"
    rel = np.zeros(24)
    for k, i in enumerate(loc):
        rel[6 * k:6 * k + 3] = x_env[i, 0:3] - x_env[j, 0:3]
        rel[6 * k + 3:6 * k + 6] = x_env[i, 7:10] - x_env[j, 7:10]
    return rel, bool(np.array_equal(got, i_ref))


def check_obs_against_own_state(dpe, kin, idx, rel, idx_base=None, what=""):
    """Observations checked against the oracle restarted from the state they describe: KIN
    carries p, q, v, omega of every drone, so the oracle recomputes roll/pitch/yaw and the
    4 nearest neighbours from it (a valid list by assert_knn_valid, features within 1e-6,
    floor 1 cm, of the drones listed).
    idx_base[e] is the global index of env e's first drone (default: CSR offsets)."""
    kin = np.asarray(kin, dtype=np.float64)
    idx = np.asarray(idx)
    rel = np.asarray(rel, dtype=np.float64)
    env_off = np.concatenate([[0], np.cumsum(dpe)])
    x = np.concatenate([kin[:, 0:7], kin[:, 10:16]], axis=1)
    for e in range(len(dpe)):
        b, N = int(env_off[e]), int(dpe[e])
        base = b if idx_base is None else int(idx_base[e])
        for j in range(N):
            k_ref = oracle.kin(x[b + j], kin[b + j, 16:20])
            assert excess(kin[b + j, 7:10], k_ref[7:10], 1e-6) <= 1.0, f"{what}: rpy of drone {b + j}"
            r_ref, _ = assert_knn_valid(x[b:b + N], j, base, idx[b + j], what=f"{what}: neighbours of drone {b + j}")
            assert excess(rel[b + j], r_ref, 1e-6, floor=1e-2) <= 1.0, f"{what}: features of drone {b + j}"


def oracle_horizon(P, dpe, flags, act_types, x0, integ0, a0, actions, n_sub, seed=0):
    """The oracle's K-step trajectory (actions [K, n, 4]) and, per step, its response to an
    initial-state error of exactly the per-substep tolerance (see tolerance_response).
    Returns (states [K, n, 13], responses [K, n, 13])."""
    env_off = np.concatenate([[0], np.cumsum(dpe)]).astype(np.int32)
    rng = np.random.default_rng(seed)
    sgn = rng.choice([-1.0, 1.0], size=x0.shape)
    x2 = x0.copy()
    for sl, tol in ((slice(0, 3), RTOL_PV), (slice(7, 10), RTOL_PV), (slice(10, 13), RTOL_W)):
        x2[:, sl] = x0[:, sl] + sgn[:, sl] * tol * np.maximum(np.abs(x0[:, sl]), 1.0)
    q = x0[:, 3:7] + sgn[:, 3:7] * ATOL_Q
    x2[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    fl = np.asarray(flags, np.int32)
    at = np.asarray(act_types, np.int32)
    xa, ia, aa = x0.copy(), integ0.copy(), a0.copy()
    xb, ib, ab = x2, integ0.copy(), a0.copy()
    states, resp = [], []
    for k in range(actions.shape[0]):
        a_k = np.asarray(actions[k], np.float64)[None]
        xa, ia, aa = oracle.control_steps(P, env_off, fl, at, xa, ia, aa, a_k, n_sub)
        xb, ib, ab = oracle.control_steps(P, env_off, fl, at, xb, ib, ab, a_k, n_sub)
        states.append(xa.copy())
        resp.append(np.abs(xa - xb))
    return np.stack(states), np.stack(resp)


def ensemble_check(snaps_a, snaps_b, alpha=1e-3):
    """Compare two trajectories of the same swarm as ensembles, snapshot by snapshot ([n, 13]
    states at the same times): per snapshot, the fraction of non-finite drones within 3
    binomial standard errors, and for height z, speed |v| and body-rate magnitude |w| of the
    finite drones a two-sample Kolmogorov-Smirnov test at level alpha / (number of tests)
    and the means within 3 standard errors. Returns (ok, first failure or '')."""
    from scipy import stats
    n_tests = 3 * len(snaps_a)
    for t, (a, b) in enumerate(zip(snaps_a, snaps_b)):
        fa, fb = np.isfinite(a).all(axis=1), np.isfinite(b).all(axis=1)
        k1, k2, n1, n2 = int((~fa).sum()), int((~fb).sum()), a.shape[0], b.shape[0]
        p = (k1 + k2) / (n1 + n2)
        se = np.sqrt(max(p * (1 - p), 1.0 / (n1 + n2)) * (1.0 / n1 + 1.0 / n2))
        if abs(k1 / n1 - k2 / n2) > 3 * se:
            return False, f"snapshot {t}: non-finite fractions {k1 / n1:.4f} vs {k2 / n2:.4f}"
        if fa.sum() < 0.5 * n1 or fb.sum() < 0.5 * n2:
            return False, f"snapshot {t}: fewer than half the drones finite"
        for name, f in (("z", lambda x: x[:, 2]), ("|v|", lambda x: np.linalg.norm(x[:, 7:10], axis=1)),
                        ("|w|", lambda x: np.linalg.norm(x[:, 10:13], axis=1))):
            g, o = f(a)[fa], f(b)[fb]
            pv = stats.ks_2samp(g, o).pvalue
            if pv <= alpha / n_tests:
                return False, f"snapshot {t} {name}: KS p = {pv:.2e}"
            se = np.sqrt(g.var(ddof=1) / g.size + o.var(ddof=1) / o.size)
            if abs(g.mean() - o.mean()) > 3 * se + 1e-12:
                return False, f"snapshot {t} {name}: means {g.mean():.6g} vs {o.mean():.6g}, 3 SE {3 * se:.3g}"
    return True, ""


def oracle_snapshots(P, swarm, act_type, actions, every, x0=None, n_sub=5):
    """The oracle's trajectory of a swarm from rest (or from x0 [n, 13]) with actions [K, n, 4],
    the state recorded every `every` control steps. Returns a list of [n, 13] states."""
    x = (np.concatenate([swarm.p, swarm.q, swarm.v, swarm.w], axis=1).astype(np.float64) if x0 is None
         else np.asarray(x0, np.float64).copy())
    integ = np.zeros((swarm.n, 6))
    a = np.zeros((swarm.n, 4))
    env_off = np.concatenate([[0], np.cumsum(swarm.drones_per_env)]).astype(np.int32)
    acts = np.full(swarm.n_envs, act_type, np.int32)
    snaps = []
    for k0 in range(0, actions.shape[0], every):
        x, integ, a = oracle.control_steps(P, env_off, np.asarray(swarm.flags, np.int32), acts, x, integ, a,
                                           np.asarray(actions[k0:k0 + every], np.float64), n_sub)
        snaps.append(x.copy())
    return snaps
