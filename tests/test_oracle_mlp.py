"""Pins for the oracle of the learned early-stop network (not from the paper; a plain MLP with a
softmax cross-entropy loss): its analytic gradient against central finite differences in FP64,
and closed forms for the loss."""
import numpy as np

import oracle


def _rand(seed=0, count=37):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(oracle.mlp_nparams()) * 0.3
    x = rng.standard_normal((count, 12)).astype(np.float32)
    y = rng.integers(0, 2, count).astype(np.int32)
    return w, x, y


def test_gradient_matches_finite_differences():
    w, x, y = _rand()
    _, g = oracle.mlp_loss_grad(w, x, y)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(w), 300, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oracle.mlp_loss_grad(wp, x, y, False) - oracle.mlp_loss_grad(wm, x, y, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_zero_weights_give_log2_loss_and_half_probability():
    # all parameters zero: z = 0 for every sample -> loss = log 2, p(stop) = 1/2, gradient only
    # on the output bias: mean(softmax - onehot) = (1/2 - frac0, 1/2 - frac1)
    _, x, y = _rand(2, 50)
    w = np.zeros(oracle.mlp_nparams())
    loss, g = oracle.mlp_loss_grad(w, x, y)
    assert abs(loss - np.log(2)) < 1e-15
    np.testing.assert_allclose(oracle.mlp_predict(w, x), 0.5)
    frac1 = y.mean()
    np.testing.assert_allclose(g[-2:], [0.5 - (1 - frac1), 0.5 - frac1], atol=1e-15)
    assert np.all(g[:-2] == 0)


def test_output_bias_alone_sets_the_probability():
    # only b3 non-zero: z = b3 -> p(stop) = sigmoid(b3[1] - b3[0])
    _, x, y = _rand(3, 10)
    w = np.zeros(oracle.mlp_nparams())
    w[-2:] = [0.25, 1.5]
    np.testing.assert_allclose(oracle.mlp_predict(w, x), 1 / (1 + np.exp(-1.25)), rtol=1e-14)


def _hand_network():
    # h1[5] = relu(x[3]), h1[9] = relu(-x[3]); h2[7] = relu(h1[5] + h1[9]) = |x3|,
    # h2[20] = relu(h1[9] - h1[5]) = relu(-x3); z[1] (stop) = 2 h2[7], z[0] (continue) = 0.5 h2[20].
    # Without the first ReLU h2[7] would be 0 and h2[20] relu(-2 x3); without the second, h2[20]
    # would be -x3. Parameters: W1 [64][12], b1, W2 [64][64], b2, W3 [2][64], b3, row-major.
    IN, H = 12, 64
    ow1, ob1 = 0, H * IN
    ow2 = ob1 + H
    ob2 = ow2 + H * H
    ow3 = ob2 + H
    w = np.zeros(oracle.mlp_nparams())
    w[ow1 + 5 * IN + 3] = 1.0
    w[ow1 + 9 * IN + 3] = -1.0
    w[ow2 + 7 * H + 5] = 1.0
    w[ow2 + 7 * H + 9] = 1.0
    w[ow2 + 20 * H + 9] = 1.0
    w[ow2 + 20 * H + 5] = -1.0
    w[ow3 + 1 * H + 7] = 2.0
    w[ow3 + 0 * H + 20] = 0.5
    return w


def test_hand_built_network_closed_form():
    # p(stop) = sigmoid(2 |x3| - 0.5 relu(-x3)): pins which input feeds which unit (W1 not
    # transposed), both ReLUs, the second layer's wiring and which output is "stop"; the loss is
    # then -log p for label 1 and -log(1 - p) for label 0.
    w = _hand_network()
    rng = np.random.default_rng(4)
    x = rng.standard_normal((64, 12)).astype(np.float32)
    x[:4, 3] = [1.5, -2.0, 0.0, 0.25]
    x3 = x[:, 3].astype(np.float64)
    t = 2.0 * np.abs(x3) - 0.5 * np.maximum(-x3, 0)
    p = 1 / (1 + np.exp(-t))
    np.testing.assert_allclose(oracle.mlp_predict(w, x), p, rtol=1e-13)
    y = rng.integers(0, 2, len(x)).astype(np.int32)
    want = np.mean(np.where(y == 1, -np.log(p), -np.log1p(-p)))
    assert abs(oracle.mlp_loss_grad(w, x, y, False) - want) < 1e-13
