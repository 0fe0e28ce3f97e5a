"""Pins of the oracle's learned-smoother network."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_is_round_to_nearest_even():
    # exactly representable values pass unchanged
    vals = np.array([1.0, -2.0, 0.5, 3.0, 0.0, 1.0 + 2 ** -7])
    assert np.array_equal(mlp.bf16(vals), vals)
    # halfway between 1 and 1 + 2^-7 rounds to even (1.0); just above rounds up
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # halfway, odd below -> up
    x = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= np.abs(x) * 2 ** -8 + 1e-300)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    W1, W2, w3 = mlp.init_weights(3)
    X = rng.normal(size=(64, 16))
    X[:, 15] = 0.0
    t = rng.normal(size=64)
    L, dW1, dW2, dw3 = mlp.loss_and_grad(W1, W2, w3, X, t)
    h = 1e-6
    for P, G in ((W1, dW1), (W2, dW2), (w3, dw3)):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, 12, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp = mlp.loss_and_grad(W1, W2, w3, X, t)[0]
            flat[idx] = old - h
            Lm = mlp.loss_and_grad(W1, W2, w3, X, t)[0]
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - G.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_network_is_positively_homogeneous_and_zero_weights_vanish():
    W1, W2, w3 = mlp.init_weights(5)
    X = np.random.default_rng(2).normal(size=(32, 16))
    out, _ = mlp.forward(W1, W2, w3, X)
    out3, _ = mlp.forward(W1, W2, w3, 3.5 * X)
    assert np.allclose(out3, 3.5 * out, rtol=1e-13)
    z = [np.zeros_like(W1), np.zeros_like(W2), np.zeros_like(w3)]
    assert np.all(mlp.forward(*z, X)[0] == 0.0)


def test_single_hidden_unit_closed_form():
    # one active path: W1 = e_0 row 0, W2 = e_00, w3 = c e_0  ->  out = c relu(x_0)
    W1 = np.zeros((32, 16)); W1[0, 0] = 1.0
    W2 = np.zeros((32, 32)); W2[0, 0] = 1.0
    w3 = np.zeros(32); w3[0] = 2.0
    X = np.array([[3.0] + [0.0] * 15, [-1.0] + [0.0] * 15])
    t = np.array([1.0, 0.5])
    out, _ = mlp.forward(W1, W2, w3, X)
    assert np.allclose(out, [6.0, 0.0])
    L, dW1, dW2, dw3 = mlp.loss_and_grad(W1, W2, w3, X, t)
    # L = ((6-1)^2 + (0-0.5)^2)/2 ; dL/dw3_0 = (2/2)*(5*3 + (-0.5)*0) = 15
    assert np.isclose(L, (25 + 0.25) / 2)
    assert np.isclose(dw3[0], 15.0)
    assert np.isclose(dW1[0, 0], (2 / 2) * 5 * 2.0 * 1.0 * 3.0)


def test_adam_first_step_is_lr_times_sign():
    """Bias-corrected Adam (Kingma & Ba 2015): after one step m_hat = g and
    v_hat = g^2, so every parameter moves by lr * sign(g) (eps negligible);
    with a constant gradient the step stays lr * sign(g)."""
    g = np.array([0.3, -2.0, 5e-3, -1e-2])
    p = np.zeros(4)
    m, v = np.zeros(4), np.zeros(4)
    lr = 1e-3
    for step in (1, 2, 3):
        before = p.copy()
        mlp.adam_step([p], [g], [m], [v], step, lr=lr, eps=1e-12)
        assert np.allclose(p - before, -lr * np.sign(g), rtol=1e-9, atol=0)
