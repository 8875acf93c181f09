"""GPU parity of the learned surrogate's BF16 tensor-core kernels against the FP64 MLP
oracle (forward, gradients, Adam), its inputs against the dynamics oracle, and the
surrogate control step: its one-step error against the plain integrator, what the network
gains over predicting no change, and the out-of-distribution fallback."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_08039_gb300 as mdg
from oracle import mlp as omlp
from paper_2606_08039_gb300 import surrogate as sg
from paper_2606_08039_gb300 import workloads as wl
from helpers import assert_horizon_close, assert_knn_valid, check_obs_against_own_state, excess, oracle_arrays, oracle_step, \
    spread_heights, tolerance_response

pytestmark = pytest.mark.gpu

P = oracle.cf2x()
HOVER = oracle.hover_rpm(P)


def _layers(seed, bias_scale=0.1):
    layers = wl.mlp_init(seed)
    out = []
    for l, (W, b) in enumerate(layers):
        bb = wl.uniform_range(-bias_scale, bias_scale, seed, wl.S_MLP, 100 + l, np.arange(b.size, dtype=np.uint64), 0)
        out.append((W, bb))
    return out


def _inputs(seed, B):
    x = np.zeros((B, mdg.MLP_IN_PAD), np.float32)
    x[:, :mdg.MLP_IN] = wl.uniform_range(-2, 2, seed, 11, 0, np.arange(B, dtype=np.uint64)[:, None],
                                         np.arange(mdg.MLP_IN, dtype=np.uint64)[None, :])
    return x


def _tanh_error_response(params, x, y_ref, rel=2.0 ** -11):
    """|change of the oracle's output| when every tanh inside SiLU = z/2 (1 + tanh(z/2))
    carries a relative error of `rel` (random signs)."""
    rng = np.random.default_rng(0)
    exact = omlp.silu

    def perturbed(z):
        return 0.5 * z * (1.0 + np.tanh(z / 2) * (1.0 + rel * rng.choice([-1.0, 1.0], size=np.shape(z))))
    omlp.silu = perturbed
    try:
        yp, _ = omlp.forward(params, x, bf16_storage=True)
    finally:
        omlp.silu = exact
    return np.abs(yp - y_ref)


def _f64(layers):
    return [(np.asarray(W, np.float64), np.asarray(b, np.float64)) for W, b in layers]


@pytest.mark.parametrize("path,B", [(mdg.MLP_PATH_TCGEN05, 128), (mdg.MLP_PATH_TCGEN05, 384 * 8),
                                    (mdg.MLP_PATH_MMA_SYNC, 384), (mdg.MLP_PATH_TCGEN05_PAIRS, 128),
                                    (mdg.MLP_PATH_TCGEN05_PAIRS, 384 * 8)])
def test_forward_matches_oracle(cuda, path, B):
    """The inference paths (fused tcgen05 kernel, its two-tiles-in-flight form, per-layer
    mma.sync GEMMs) against the oracle on identical bf16 inputs and weights; several tiles per
    block for the persistent tcgen05 kernels, and for the paired one a lone tile."""
    layers = _layers(1)
    m = mdg.MLP(B, layers)
    m.set_path(path)
    x = torch.as_tensor(_inputs(2, B), device=cuda).to(torch.bfloat16)
    y = torch.full((B, mdg.MLP_OUT_PAD), float("nan"), device=cuda)
    m.forward(x, y)
    torch.cuda.synchronize()
    assert m.status() == 0
    xo = x.float().cpu().numpy().astype(np.float64)
    yo, _ = omlp.forward(_f64(layers), xo, bf16_storage=True)
    # identical bf16 inputs and weights; FP32 vs FP64 accumulation can flip the bf16 rounding
    # of a hidden activation by one bf16 unit (2^-8 relative), hence 1e-2 max(|y|, 1). The
    # tcgen05 path evaluates SiLU as z/2 (1 + tanh(z/2)) with tanh.approx.f32 (relative error
    # 2^-11): its bound adds the oracle's own response to that error.
    bound = 1e-2 * np.maximum(np.abs(yo), 1.0)
    if path != mdg.MLP_PATH_MMA_SYNC:
        bound = bound + _tanh_error_response(_f64(layers), xo, yo)
    assert np.all(np.abs(y.cpu().numpy() - yo) <= bound)


def test_training_paths_agree_over_steps(cuda):
    """Eight Adam steps on the tcgen05 path and on the mma.sync path from the same weights and
    batches: losses within 1% and the weights within 10% of their change (accumulation order
    and bf16 rounding of the stored activations differ, and Adam's first steps move a weight
    by about lr whatever the size of its gradient, so the sign of a near-zero gradient
    matters)."""
    B = 512
    layers = _layers(7)
    x = torch.as_tensor(_inputs(8, B), device=cuda).to(torch.bfloat16)
    t = torch.zeros((B, mdg.MLP_OUT_PAD), device=cuda)
    t[:, :mdg.MLP_OUT] = torch.as_tensor(
        wl.uniform_range(-1, 1, 9, 12, 0, np.arange(B, dtype=np.uint64)[:, None],
                         np.arange(mdg.MLP_OUT, dtype=np.uint64)[None, :]), device=cuda)
    w0 = mdg.mlp_flatten(layers).astype(np.float64)
    out = []
    for path in (mdg.MLP_PATH_TCGEN05, mdg.MLP_PATH_MMA_SYNC):
        m = mdg.MLP(B, layers)
        m.set_train_path(path)
        loss = torch.zeros(1, device=cuda)
        losses = []
        for _ in range(8):
            m.grad(x, t, loss)
            losses.append(float(loss))
            m.adam(1e-3)
        torch.cuda.synchronize()
        assert m.status() == 0
        out.append((np.array(losses), m.params().astype(np.float64)))
    (la, wa), (lb, wb) = out
    np.testing.assert_allclose(la, lb, rtol=1e-2)
    assert la[-1] < la[0]
    dw = np.abs(wb - w0)
    assert np.linalg.norm(wa - wb) <= 0.1 * np.linalg.norm(dw)


@pytest.mark.parametrize("path", [mdg.MLP_PATH_TCGEN05, mdg.MLP_PATH_TCGEN05_PAIRS])
def test_tcgen05_bounded_wait_exit(cuda, path):
    """The tcgen05 kernel's exit on an expired wait, without a stuck device: with wait bounds
    of zero the first wait that is not already complete (at the latest the epilogue's wait
    for its first accumulator) gives up on a normal 256-row launch, in both tcgen05 kernels. The launch returns with
    MDG_STATUS_TIMEOUT set; a launch with the default bounds then matches the oracle, so the
    abandoned launch drained its copies and MMAs and freed its tensor memory."""
    layers = _layers(1)
    B = 256  # one pair of tiles for the paired kernel
    m = mdg.MLP(B, layers)
    m.set_path(path)
    x = torch.as_tensor(_inputs(2, B), device=cuda).to(torch.bfloat16)
    y = torch.full((B, mdg.MLP_OUT_PAD), float("nan"), device=cuda)
    m.set_wait_limits(0, 0)
    m.forward(x, y)
    assert mdg.lib().mdg_sync(mdg._stream(None), 5000) == mdg.OK  # the launch returned
    assert m.status() & mdg.STATUS_TIMEOUT
    for _ in range(2):  # again, and on the blocks' second use of the SMs' tensor memory
        m.forward(x, y)
        torch.cuda.synchronize()
        assert m.status() & mdg.STATUS_TIMEOUT
    m.set_wait_limits()
    y.fill_(float("nan"))
    m.forward(x, y)
    torch.cuda.synchronize()
    assert m.status() == 0
    xo = x.float().cpu().numpy().astype(np.float64)
    yo, _ = omlp.forward(_f64(layers), xo, bf16_storage=True)
    bound = 1e-2 * np.maximum(np.abs(yo), 1.0) + _tanh_error_response(_f64(layers), xo, yo)
    assert np.all(np.abs(y.cpu().numpy() - yo) <= bound)


@pytest.mark.parametrize("n_tiles", [305, 611])
def test_paired_kernel_equals_single_tile_kernel(cuda, n_tiles):
    """The two-tiles-in-flight kernel does the first tile of each pair (A, even tiles) exactly
    as the single-tile kernel (the same MMAs in the same order, the same epilogue per element),
    so those outputs are bit-identical; the second tile (B) sums the K chunks of its hidden
    layers in the order 3, 2, 1, 0, so it agrees to FP32 summation order (and the bf16
    rounding that follows). Here with two to three pairs per block and a lone last tile (305
    tiles: 153 pairs on 152 SMs; 611 tiles); and sampled tiles of it against the oracle."""
    B = 128 * n_tiles
    layers = _layers(4)
    m = mdg.MLP(B, layers)
    x = torch.as_tensor(_inputs(6, B), device=cuda).to(torch.bfloat16)
    ys = []
    for path in (mdg.MLP_PATH_TCGEN05, mdg.MLP_PATH_TCGEN05_PAIRS):
        m.set_path(path)
        y = torch.full((B, mdg.MLP_OUT_PAD), float("nan"), device=cuda)
        m.forward(x, y)
        torch.cuda.synchronize()
        assert m.status() == 0
        ys.append(y)
    single, paired = (y.view(n_tiles, 128, mdg.MLP_OUT_PAD) for y in ys)
    assert torch.equal(single[0::2], paired[0::2])
    assert torch.all((single[1::2] - paired[1::2]).abs() <= 1e-2 * torch.clamp(single[1::2].abs(), min=1.0))
    tiles = [0, 1, 151, 152, 153, 303, 304, n_tiles - 2, n_tiles - 1]
    rows = np.concatenate([np.arange(128 * t, 128 * t + 128) for t in sorted(set(tiles))])
    xo = x[torch.as_tensor(rows, device=cuda)].float().cpu().numpy().astype(np.float64)
    yo, _ = omlp.forward(_f64(layers), xo, bf16_storage=True)
    bound = 1e-2 * np.maximum(np.abs(yo), 1.0) + _tanh_error_response(_f64(layers), xo, yo)
    assert np.all(np.abs(ys[1].cpu().numpy()[rows] - yo) <= bound)


@pytest.mark.parametrize("path,B", [(mdg.MLP_PATH_TCGEN05, 256), (mdg.MLP_PATH_TCGEN05, 1024),
                                    (mdg.MLP_PATH_MMA_SYNC, 256)])
def test_gradients_and_loss_match_oracle(cuda, path, B):
    """Loss and every gradient of both training paths (tcgen05 with TMEM accumulators, the
    default; mma.sync) against the FP64 oracle's backward on the same bf16 tensors; B = 1024
    splits the weight gradients over the batch (two slices added with atomics)."""
    layers = _layers(3)
    m = mdg.MLP(B, layers)
    m.set_train_path(path)
    x = torch.as_tensor(_inputs(4, B), device=cuda).to(torch.bfloat16)
    t = np.zeros((B, mdg.MLP_OUT_PAD), np.float32)
    t[:, :mdg.MLP_OUT] = wl.uniform_range(-1, 1, 5, 12, 0, np.arange(B, dtype=np.uint64)[:, None],
                                          np.arange(mdg.MLP_OUT, dtype=np.uint64)[None, :])
    loss = torch.zeros(1, device=cuda)
    m.grad(x, torch.as_tensor(t, device=cuda), loss)
    torch.cuda.synchronize()
    g = mdg.mlp_unflatten(m.grads())
    # the oracle network with the 13 used outputs
    p13 = _f64(layers)
    p13[3] = (p13[3][0][:mdg.MLP_OUT], p13[3][1][:mdg.MLP_OUT])
    xo = x.float().cpu().numpy().astype(np.float64)
    yo, cache = omlp.forward(p13, xo, bf16_storage=True)
    go = omlp.backward(p13, cache, yo, t[:, :mdg.MLP_OUT].astype(np.float64), bf16_storage=True)
    assert float(loss) == pytest.approx(omlp.mse(yo, t[:, :mdg.MLP_OUT]), rel=1e-3)
    for l in range(4):
        gw, gb = g[l]
        if l == 3:
            assert np.all(gw[mdg.MLP_OUT:] == 0) and np.all(gb[mdg.MLP_OUT:] == 0)
            gw, gb = gw[:mdg.MLP_OUT], gb[:mdg.MLP_OUT]
        for a, b in ((gw, go[l][0]), (gb, go[l][1])):
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel < 2e-2, f"layer {l}: relative gradient error {rel:.3g}"
    assert np.all(g[0][0][:, mdg.MLP_IN:] == 0)  # padded inputs get no gradient


def test_adam_matches_oracle(cuda):
    B = 128
    layers = _layers(6)
    m = mdg.MLP(B, layers)
    x = torch.as_tensor(_inputs(7, B), device=cuda).to(torch.bfloat16)
    t = torch.zeros((B, mdg.MLP_OUT_PAD), device=cuda)
    t[:, :mdg.MLP_OUT] = 0.5
    params = _f64(mdg.mlp_unflatten(m.params()))
    mo, vo = omlp.adam_init(params)
    for step in (1, 2, 3):
        m.grad(x, t)
        torch.cuda.synchronize()
        grads = _f64(mdg.mlp_unflatten(m.grads()))
        m.adam(1e-3)
        torch.cuda.synchronize()
        params, mo, vo = omlp.adam_step(params, grads, mo, vo, step, lr=1e-3)
        got = mdg.mlp_unflatten(m.params())
        for (Wg, bg), (Wo, bo) in zip(got, params):
            np.testing.assert_allclose(Wg, Wo, rtol=1e-5, atol=1e-7)
            np.testing.assert_allclose(bg, bo, rtol=1e-5, atol=1e-7)


def test_training_reduces_the_loss(cuda):
    B, rows = 512, 4096
    teacher = _f64(_layers(8, bias_scale=0.5))
    teacher[3] = (teacher[3][0][:mdg.MLP_OUT] * 0.3, teacher[3][1][:mdg.MLP_OUT])
    xn = _inputs(9, rows)
    yt, _ = omlp.forward(teacher, xn.astype(np.float64))
    t = np.zeros((rows, mdg.MLP_OUT_PAD), np.float32)
    t[:, :mdg.MLP_OUT] = (yt - yt.mean(0)) / yt.std(0)
    m = mdg.MLP(B, wl.mlp_init(10))
    x = torch.as_tensor(xn, device=cuda).to(torch.bfloat16)
    tt = torch.as_tensor(t, device=cuda)
    loss = torch.zeros(1, device=cuda)
    first = None
    for it in range(400):
        sl = slice((it % (rows // B)) * B, (it % (rows // B) + 1) * B)
        m.grad(x[sl].contiguous(), tt[sl].contiguous(), loss)
        if first is None:
            first = float(loss)
        m.adam(2e-3)
    torch.cuda.synchronize()
    assert float(loss) < 0.1 * first


def test_features_match_state_and_oracle_neighbours(cuda):
    sw = wl.full_aero(13, n_envs=150)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    rpm = torch.as_tensor(wl.rpm_actions(13, sw.n, 0, HOVER), device=cuda)
    raw = torch.empty((sw.n, mdg.MLP_IN), device=cuda)
    h.features(state, rpm, raw)
    torch.cuda.synchronize()
    raw = raw.cpu().numpy()
    x, _, _ = oracle_arrays(state)
    np.testing.assert_array_equal(raw[:, :13], x.astype(np.float32))
    np.testing.assert_array_equal(raw[:, 13:17], rpm.cpu().numpy())
    env_off = sw.env_off
    for e in range(sw.n_envs):
        b, N = int(env_off[e]), int(sw.drones_per_env[e])
        xe = x[b:b + N]
        for j in range(N):
            # the drone each listed slot describes (the one whose relative position it holds),
            # then that list checked as a valid 4-nearest list and the features against it
            listed = np.full(4, -1)
            for k in range(min(4, N - 1)):
                dp = np.abs(xe[:, 0:3] - xe[j, 0:3] - raw[b + j, 17 + 6 * k:20 + 6 * k]).sum(axis=1)
                dp[j] = np.inf
                listed[k] = b + int(np.argmin(dp))
            r_ref, _ = assert_knn_valid(xe, j, b, listed, what=f"features of drone {b + j}")
            assert excess(raw[b + j, 17:], r_ref, 1e-6, floor=1e-2) <= 1.0


@pytest.fixture(scope="module")
def trained(cuda):
    raw, delta = sg.generate_transitions(4096, 24, seed=21, device=cuda)
    data = sg.Dataset(raw, delta)
    m = mdg.MLP(8192, wl.mlp_init(22))
    data.attach(m)
    hist = sg.fit(m, data, epochs=6, batch=8192, lr=2e-3)
    return m, data, hist


def test_surrogate_step_gains_over_no_network(cuda, trained):
    m, data, hist = trained
    assert hist[-1] < 0.5 * hist[0]
    sw = wl.full_aero(77, n_envs=1024)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    s_sur = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    s_pln = s_sur.clone()
    before = sg.state13(s_sur).clone()
    wp = torch.as_tensor(wl.waypoints(77, sw.n), device=cuda)
    nfb = torch.zeros(1, dtype=torch.int32, device=cuda)
    m.step(h, s_sur, wp, mdg.ACT_PID, 5, 4.0, nfb)
    h.step(s_pln, wp, mdg.ACT_PID, 5)
    torch.cuda.synchronize()
    xs, xp = sg.state13(s_sur), sg.state13(s_pln)
    true_d = xp - before
    n_fb = int(nfb)
    assert n_fb < 0.5 * sw.n_envs
    # Evaluate where the network is meant to work: drones not sent to the integrator whose
    # true state change lies in the regular regime the network was trained on (standardised
    # change within +-8); the rest is the chaotic tail of near-coincident heights.
    zt = (true_d - data.out_mean) / data.out_std
    diff = (xs - xp).abs().max(dim=1).values
    env_fb = (diff.view(-1, 4) == 0).all(dim=1).repeat_interleave(4)  # fallback envs match the plain step
    regular = (zt.abs() <= 8).all(dim=1) & ~env_fb
    assert float(regular.float().mean()) > 0.5
    # One-step error of the surrogate vs the plain integrator against the error of a
    # predictor without the network (state unchanged). The rotational change depends on
    # the motor torques alone and is learned closely (this small training: 0.22 quaternion,
    # 0.085 body rate). The translational change is dominated by the downwash law's 1/dz^2:
    # the formation's drones fly at nearly equal heights (median 1.1 cm to the nearest other
    # height), which the network does not represent; velocity is required to gain (0.955
    # measured), position only not to lose more than 10% (1.06 measured: the network's
    # spurious vertical motion costs about what it gains).
    for name, sl, bound in (("quaternion", slice(3, 7), 0.3), ("body rate", slice(10, 13), 0.3),
                            ("position", slice(0, 3), 1.1), ("velocity", slice(7, 10), 1.0)):
        err = (xs[regular, sl] - xp[regular, sl]).pow(2).mean().sqrt()
        base = true_d[regular, sl].pow(2).mean().sqrt()
        assert err < bound * base, f"{name}: surrogate rms error {float(err):.3g} vs no-network {float(base):.3g}"
    # quaternions stay unit
    q = xs[:, 3:7]
    assert torch.allclose(q.norm(dim=1), torch.ones_like(q[:, 0]), atol=1e-5)


def test_out_of_distribution_environments_take_the_integrator(cuda, trained):
    m, data, _ = trained
    sw = wl.full_aero(78, n_envs=300)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    wp = wl.waypoints(78, sw.n)
    nfb = torch.zeros(1, dtype=torch.int32, device=cuda)
    m.step(h, state, torch.as_tensor(wp, device=cuda), mdg.ACT_PID, 5, 0.0, nfb)  # everything out of distribution
    torch.cuda.synchronize()
    assert int(nfb) == sw.n_envs
    xg, ig, _ = oracle_arrays(state)
    layout = (sw.drones_per_env, sw.flags)
    acts = np.full(sw.n_envs, mdg.ACT_PID)
    xo, io, _ = oracle_step(P, layout, x0, i0, a0, wp, acts, 5)
    resp = tolerance_response(P, layout, x0, i0, a0, wp, acts, 5)
    assert_horizon_close(xg, xo, resp, 5, what="fallback")
    assert excess(ig, io, 1e-5) <= 1.0
    assert h.status()[0] == mdg.OK


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_fallback_of_large_environments(cuda, trained, integrator):
    """Environments of 64 drones (the dense swarm's size, one block per environment in the
    fallback) and Runge-Kutta substeps: with every environment out of distribution the
    surrogate step is the plain integrator, against the oracle over the control step (heights
    spread per environment, so that the downwash is well conditioned)."""
    m, data, _ = trained
    sw = spread_heights(wl.dense(80, n_envs=24), dz=0.3, z0=0.5)
    c = mdg.Constants.cf2x()
    Po = oracle.cf2x()
    if integrator == "rk4":
        c.integrator = mdg.INTEGRATOR_RK4
        Po.integrator = oracle.RK4
    h = mdg.Handle(sw.drones_per_env, sw.flags, c)
    state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    x0, i0, a0 = oracle_arrays(state)
    act = wl.rpm_actions(80, sw.n, 0, HOVER)
    nfb = torch.zeros(1, dtype=torch.int32, device=cuda)
    m.step(h, state, torch.as_tensor(act, device=cuda), mdg.ACT_RPM, 5, 0.0, nfb)
    torch.cuda.synchronize()
    assert int(nfb) == sw.n_envs
    xg, _, ag = oracle_arrays(state)
    layout = (sw.drones_per_env, sw.flags)
    acts = np.full(sw.n_envs, mdg.ACT_RPM)
    xo, _, ao = oracle_step(Po, layout, x0, i0, a0, act, acts, 5)
    resp = tolerance_response(Po, layout, x0, i0, a0, act, acts, 5)
    assert_horizon_close(xg, xo, resp, 5, what=f"fallback of 64-drone environments ({integrator})")
    np.testing.assert_allclose(ag, ao, rtol=1e-6)
    assert h.status()[0] == mdg.OK


def test_surrogate_step_paths_agree(cuda, trained):
    m, data, _ = trained
    sw = wl.full_aero(79, n_envs=512)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    wp = torch.as_tensor(wl.waypoints(79, sw.n), device=cuda)
    out = []
    for path in (mdg.MLP_PATH_MMA_SYNC, mdg.MLP_PATH_TCGEN05, mdg.MLP_PATH_TCGEN05_PAIRS):
        m.set_path(path)
        st = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
        m.step(h, st, wp, mdg.ACT_PID, 5, 4.0)
        torch.cuda.synchronize()
        out.append(sg.state13(st).cpu().numpy().astype(np.float64))
    m.set_path(mdg.MLP_PATH_TCGEN05_PAIRS)  # the default
    # same network, same inputs and the same out-of-distribution decisions: the states differ
    # only by out_std times the difference of the standardised outputs, which the forward
    # test bounds by 1e-2 max(|y|, 1); |y| stays below ~4 in distribution, hence 0.05 out_std
    tol = 0.05 * data.out_std.cpu().numpy().astype(np.float64)
    for o in out[1:]:
        assert np.all(np.abs(o - out[0]) <= tol[None, :])
    assert h.status()[0] == mdg.OK


def test_transition_is_features_then_step(cuda):
    """mdg_transition: the applied RPMs are rpm times rpm_scale, the inputs are mdg_features of
    the state with them, the state advances by mdg_step, and delta is after minus before."""
    sw = wl.full_aero(14, n_envs=200)
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    s_a = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
    s_b = s_a.clone()
    rpm = torch.as_tensor(wl.rpm_actions(14, sw.n, 0, HOVER), device=cuda)
    scale = torch.as_tensor(wl.uniform_range(0.9, 1.1, 14, 13, 0, np.arange(sw.n, dtype=np.uint64)[:, None],
                                             np.arange(4, dtype=np.uint64)[None, :]), device=cuda)
    applied = torch.empty_like(rpm)
    raw = torch.empty((sw.n, mdg.MLP_IN), device=cuda)
    delta = torch.empty((sw.n, mdg.MLP_OUT), device=cuda)
    h.transition(s_a, rpm, applied, raw, delta, rpm_scale=scale)
    ref_rpm = rpm * scale
    raw_b = torch.empty_like(raw)
    before = sg.state13(s_b).clone()
    h.features(s_b, ref_rpm, raw_b)
    h.step(s_b, ref_rpm, mdg.ACT_RPM, 5)
    torch.cuda.synchronize()
    assert torch.equal(applied, ref_rpm)
    assert torch.equal(raw, raw_b) and torch.equal(s_a, s_b)
    assert torch.equal(delta, sg.state13(s_b) - before)


def test_fit_normalization_matches_its_definition(cuda):
    """mdg_mlp_fit_normalization against the same steps in numpy (float64): non-finite rows
    dropped; per column the 0.5% / 99.5% quantiles (linear interpolation) of an evenly strided
    sample, widened by 10% of their distance, as the trim box; FP64 mean and unbiased standard
    deviation of the kept rows (scale 1 for a constant column); rows with a standardised input
    beyond +-4 or target beyond +-8 dropped; the kept inputs' range widened by 10% plus 1e-6 as
    the out-of-distribution box; the standardised rows in order, truncated to a multiple of 128."""
    rng = np.random.default_rng(5)
    N = 300_000  # above the 262144-row sample: stride 1 (the stride is 2 only from 524288 rows)
    raw = rng.standard_normal((N, mdg.MLP_IN)).astype(np.float32) * np.linspace(0.1, 3, mdg.MLP_IN)[None, :].astype(np.float32)
    delta = rng.standard_normal((N, mdg.MLP_OUT)).astype(np.float32)
    raw[:, 5] = 2.5  # a constant column
    heavy = rng.random(N) < 0.01  # a heavy tail the trim removes
    delta[heavy, 3] *= 1e3
    raw[rng.integers(0, N, 50), 7] = np.nan
    delta[rng.integers(0, N, 50), 2] = np.inf
    m = mdg.MLP(128)
    x = torch.empty((N, mdg.MLP_IN_PAD), dtype=torch.bfloat16, device=cuda)
    t = torch.empty((N, mdg.MLP_OUT_PAD), device=cuda)
    n_fin, n_kept = m.fit_normalization(torch.as_tensor(raw, device=cuda), torch.as_tensor(delta, device=cuda), x, t)
    in_mean, in_std, out_mean, out_std, in_lo, in_hi = m.normalization()
    # the definition, in numpy
    A = np.concatenate([raw, delta], 1).astype(np.float64)
    fin = np.isfinite(A).all(1)
    F = A[fin]
    assert n_fin == F.shape[0]
    stride = max(1, F.shape[0] // 262144)
    S = F[::stride]
    qlo, qhi = np.quantile(S, 0.005, axis=0), np.quantile(S, 0.995, axis=0)
    r = qhi - qlo
    keep1 = ((F >= qlo - 0.1 * r) & (F <= qhi + 0.1 * r)).all(1)
    K1 = F[keep1]
    mean = K1.mean(0)
    sd = K1.std(0, ddof=1)
    sd = np.where(sd > 1e-6 * np.maximum(np.abs(mean), 1.0), sd, 1.0)
    np.testing.assert_allclose(in_mean, mean[:mdg.MLP_IN], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(out_mean, mean[mdg.MLP_IN:], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(in_std, sd[:mdg.MLP_IN], rtol=1e-5)
    np.testing.assert_allclose(out_std, sd[mdg.MLP_IN:], rtol=1e-5)
    assert in_std[5] == 1.0
    Z = (K1 - mean) / sd
    keep2 = (np.abs(Z[:, :mdg.MLP_IN]) <= 4.0).all(1) & (np.abs(Z[:, mdg.MLP_IN:]) <= 8.0).all(1)
    K2 = K1[keep2]
    assert abs(K2.shape[0] // 128 * 128 - n_kept) <= 128  # boundary rows may round either way in float32
    lo, hi = K2[:, :mdg.MLP_IN].min(0), K2[:, :mdg.MLP_IN].max(0)
    pad = 0.1 * (hi - lo) + 1e-6
    np.testing.assert_allclose(in_lo, lo - pad, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(in_hi, hi + pad, rtol=1e-5, atol=1e-5)
    # the emitted rows: the kept rows in order, standardised
    xs = x[:n_kept].float().cpu().numpy()
    ts = t[:n_kept].cpu().numpy()
    n_cmp = min(n_kept, K2.shape[0]) // 2  # rows before any boundary difference
    zin = (K2[:n_cmp, :mdg.MLP_IN] - mean[:mdg.MLP_IN]) / sd[:mdg.MLP_IN]
    np.testing.assert_allclose(xs[:n_cmp, :mdg.MLP_IN], zin, rtol=1e-2, atol=1e-2)
    assert np.all(xs[:, mdg.MLP_IN:] == 0) and np.all(ts[:, mdg.MLP_OUT:] == 0)
    np.testing.assert_allclose(ts[:n_cmp, :mdg.MLP_OUT], Z[keep2][:n_cmp, mdg.MLP_IN:], rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("recipe", ["full_aero", "full_aero_ragged", "dense", "dense_pid"])
def test_surrogate_step_composes_its_parts(cuda, trained, recipe):
    """mdg_surrogate_step equals its parts called one by one: the plain integrator's inputs of
    the state and its RPMs (mdg_transition), their standardisation (mdg_mlp_standardize), the
    network (mdg_mlp_forward) and the de-standardised change added on the host (quaternion
    renormalised), on 4-drone (PID; also a drone count that is not a multiple of 128) and
    64-drone (RPM and PID) environments. With the trained box every
    environment with an input outside it is counted for the fallback; with an unbounded box
    none is, and every drone is compared."""
    _, data, _ = trained
    # full_aero_ragged: 1204 drones, not a multiple of the network's 128-row tiles: the last
    # tile holds padding rows, which the fused update must not write (a row past the end of a
    # state plane is the next plane's first drone, compared below)
    sw = (wl.full_aero(81, n_envs=256) if recipe == "full_aero" else
          wl.full_aero(83, n_envs=301) if recipe == "full_aero_ragged" else wl.dense(82, n_envs=16))
    h = mdg.Handle(sw.drones_per_env, sw.flags)
    if recipe == "dense":
        action, act = torch.as_tensor(wl.rpm_actions(82, sw.n, 0, HOVER), device=cuda), mdg.ACT_RPM
    else:
        action, act = torch.as_tensor(wl.waypoints(81, sw.n), device=cuda), mdg.ACT_PID
    in_mean, in_std, out_mean, out_std, in_lo, in_hi = data.stats()
    for bounded in (True, False):
        m = mdg.MLP((sw.n + 127) // 128 * 128, wl.mlp_init(23))
        lo, hi = (in_lo, in_hi) if bounded else (np.full_like(in_lo, -1e30), np.full_like(in_hi, 1e30))
        m.set_normalization(in_mean, in_std, out_mean, out_std, lo, hi)
        ood_z = 4.0 if bounded else 1e30
        state = mdg.pack_state(sw.p, sw.q, sw.v, sw.w, device=cuda)
        before = state.clone()
        nfb = torch.zeros(1, dtype=torch.int32, device=cuda)
        m.step(h, state, action, act, 5, ood_z, nfb)
        # the parts: RPMs (the PID on a copy of the state), inputs, standardisation, network
        s2 = before.clone()
        rpm = torch.empty((sw.n, 4), device=cuda)
        if act == mdg.ACT_PID:
            h.pid(s2, action, rpm)
        else:
            rpm.copy_(action.clamp(0.0, mdg.Constants.cf2x().max_rpm()))
        raw = torch.empty((sw.n, mdg.MLP_IN), device=cuda)
        delta = torch.empty((sw.n, mdg.MLP_OUT), device=cuda)
        applied = torch.empty((sw.n, 4), device=cuda)
        h.transition(s2.clone(), rpm, applied, raw, delta)
        rows = (sw.n + 127) // 128 * 128
        x = torch.zeros((rows, mdg.MLP_IN_PAD), dtype=torch.bfloat16, device=cuda)
        m.standardize(raw, x[:sw.n])
        y = torch.empty((rows, mdg.MLP_OUT_PAD), device=cuda)
        m.forward(x, y)
        torch.cuda.synchronize()
        rawn = raw.cpu().numpy().astype(np.float64)
        z = (rawn - in_mean) / in_std
        bad = ~((np.abs(z) <= ood_z) & (rawn >= lo) & (rawn <= hi))
        env_bad = bad.reshape(sw.n_envs, -1).any(axis=1)
        assert int(nfb) == int(env_bad.sum()), (int(nfb), int(env_bad.sum()))
        if bounded:
            continue
        assert int(nfb) == 0
        d = y[:sw.n, :mdg.MLP_OUT].double().cpu().numpy() * out_std + out_mean
        x0 = sg.state13(before).double().cpu().numpy()
        want = x0 + d
        want[:, 3:7] /= np.linalg.norm(want[:, 3:7], axis=1, keepdims=True)
        got = sg.state13(state).double().cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-5 * np.maximum(np.abs(want), 1.0)), np.abs(got - want).max()
