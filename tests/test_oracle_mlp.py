"""Pins for the FP64 reference of the learned scorer (no GPU)."""
import numpy as np

from oracle import mlp


def random_params(seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.5, mlp.N_PARAMS)


def test_bf16_rounding_matches_definition():
    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(np.float32(1 + 2 ** -8))[()] == 1.0
    assert mlp.bf16(np.float32(1 + 3 * 2 ** -8))[()] == 1 + 2 ** -6
    assert mlp.bf16(np.float32(1 + 2 ** -7))[()] == 1 + 2 ** -7
    x = np.random.default_rng(1).normal(size=1000).astype(np.float32)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-45)
    np.testing.assert_array_equal(mlp.bf16(r), r)          # idempotent


def test_zero_network_outputs_the_output_bias():
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 0.75
    np.testing.assert_array_equal(mlp.forward(p, np.ones((5, 8))), 0.75)


def test_hand_computed_example():
    p = np.zeros(mlp.N_PARAMS)
    W1, b1, w2, b2 = mlp.unpack(p, False)
    # hidden 0 = relu(x0 + 2 x1 - 1), hidden 1 = relu(-x0), y = 3 h0 - 2 h1 + 0.5
    p[0], p[1] = 1.0, 2.0
    p[mlp.N_IN] = -1.0
    o_b1 = mlp.N_HID * mlp.N_IN
    p[o_b1] = -1.0
    o_w2 = o_b1 + mlp.N_HID
    p[o_w2], p[o_w2 + 1] = 3.0, -2.0
    p[-1] = 0.5
    X = np.array([[1.0, 1.0] + [0] * 6, [-2.0, 0.0] + [0] * 6])
    # row 0: h0 = 2, h1 = 0 -> 6.5; row 1: h0 = relu(-3) = 0, h1 = 2 -> -3.5
    np.testing.assert_allclose(mlp.forward(p, X, bf16_inputs=False), [6.5, -3.5])


def test_gradient_matches_finite_differences():
    p = random_params(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(40, 8))
    y = rng.normal(size=40)
    g, loss = mlp.mse_gradients(p, X, y, bf16_inputs=False)
    h = 1e-6
    for i in rng.choice(mlp.N_PARAMS, 60, replace=False).tolist() + [mlp.N_PARAMS - 1]:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        lp = np.mean((mlp.forward(p + e, X, False) - y) ** 2)
        lm = np.mean((mlp.forward(p - e, X, False) - y) ** 2)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-5 * max(1.0, abs(g[i])), i
    assert loss == np.mean((mlp.forward(p, X, False) - y) ** 2)
