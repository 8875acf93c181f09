"""Pins of the FP64 MLP oracle (oracle/mlp.py): central finite differences against the
backward pass, SiLU values and derivative, Adam's first step in closed form, a linear
special case that must converge to the least-squares solution, and bfloat16 rounding on
exactly representable cases. CPU only."""
import numpy as np
import pytest

from oracle import mlp


def _net(rng, dims):
    return [(rng.normal(size=(o, i)) / np.sqrt(i), rng.normal(size=o) * 0.1) for i, o in zip(dims[:-1], dims[1:])]


def test_backward_matches_central_finite_differences():
    rng = np.random.default_rng(0)
    params = _net(rng, [5, 7, 6, 3])
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 3))
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.mse(mlp.forward(params, x)[0], t)
                arr[idx] = old - h
                lm = mlp.mse(mlp.forward(params, x)[0], t)
                arr[idx] = old
                assert g[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)


def test_silu_values_and_derivative():
    assert mlp.silu(0.0) == 0.0 and mlp.silu_grad(0.0) == 0.5
    z = np.linspace(-8, 8, 33)
    np.testing.assert_allclose(mlp.silu(z), z * (0.5 * (1 + np.tanh(z / 2))), rtol=1e-13, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)
    # large |z|: silu -> z for z >> 0, -> 0 for z << 0; its slope -> 1 and 0
    assert mlp.silu_grad(40.0) == pytest.approx(1.0) and abs(mlp.silu_grad(-40.0)) < 1e-15


def test_adam_first_step_is_lr_times_sign():
    # after one step m_hat = g and v_hat = g^2, so the update is -lr g / (|g| + eps)
    rng = np.random.default_rng(1)
    params = _net(rng, [4, 3])
    grads = [(rng.normal(size=(3, 4)), rng.normal(size=3))]
    m, v = mlp.adam_init(params)
    new, m1, v1 = mlp.adam_step(params, grads, m, v, 1, lr=0.01)
    for (W0, b0), (W1, b1), (gW, gb) in zip(params, new, grads):
        np.testing.assert_allclose(W1 - W0, -0.01 * gW / (np.abs(gW) + 1e-8), rtol=1e-12)
        np.testing.assert_allclose(b1 - b0, -0.01 * gb / (np.abs(gb) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1[0][0], 0.1 * grads[0][0])
    np.testing.assert_allclose(v1[0][0], 0.001 * grads[0][0] ** 2)


def test_linear_model_converges_to_least_squares():
    # one linear layer: minimising the MSE is ordinary least squares with an intercept
    rng = np.random.default_rng(2)
    X = rng.normal(size=(200, 4))
    Wt = rng.normal(size=(2, 4))
    T = X @ Wt.T + np.array([0.5, -1.0]) + 0.1 * rng.normal(size=(200, 2))
    params = [(np.zeros((2, 4)), np.zeros(2))]
    m, v = mlp.adam_init(params)
    for step in range(1, 4001):
        y, cache = mlp.forward(params, X)
        params, m, v = mlp.adam_step(params, mlp.backward(params, cache, y, T), m, v, step, lr=0.01)
    A = np.hstack([X, np.ones((200, 1))])
    sol, *_ = np.linalg.lstsq(A, T, rcond=None)
    np.testing.assert_allclose(params[0][0], sol[:4].T, atol=1e-4)
    np.testing.assert_allclose(params[0][1], sol[4], atol=1e-4)


def test_bf16_rounding():
    one = 1.0
    ulp = 2.0 ** -7  # bfloat16 spacing at 1
    assert mlp.bf16(one) == one
    assert mlp.bf16(one + ulp / 2) == one            # halfway: ties to even (1.0)
    assert mlp.bf16(one + 3 * ulp / 2) == one + 2 * ulp  # halfway: ties to even (1 + 2 ulp)
    assert mlp.bf16(one + 0.75 * ulp) == one + ulp
    assert mlp.bf16(-2.5) == -2.5
    # 8 significant bits: the rounding error is at most half a unit, 2^-8 relative
    x = np.random.default_rng(3).normal(size=1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2.0 ** -8)
