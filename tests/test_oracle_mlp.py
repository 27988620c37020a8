"""CPU pins of the oracle's MLP (the learned preconditioner's network)."""
import numpy as np

from oracle import mlp


def _theta(rng, scale=0.4):
    return rng.standard_normal(mlp.N_PARAMS) * scale


def test_parameter_count():
    assert mlp.N_PARAMS == 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1 == 4609


def test_zero_weights_give_the_constant_b3():
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = 1.25
    X = np.random.default_rng(0).standard_normal((7, 5))
    g, _, _ = mlp.forward(theta, X)
    assert np.allclose(g, 1.25)


def test_single_hidden_path_closed_form():
    # only W1[0,0], W2[0,0], W3[0] non-zero: g = w3 tanh(w2 tanh(w1 x0)) + b3
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    w1, w2, w3, b3 = 0.7, -1.3, 0.9, 0.2
    theta[0] = w1                                    # W1[0, 0]
    theta[64 * 5 + 64] = w2                          # W2[0, 0]
    theta[64 * 5 + 64 + 64 * 64 + 64] = w3           # W3[0]
    theta[-1] = b3
    X = np.random.default_rng(1).standard_normal((5, 5))
    g, _, _ = mlp.forward(theta, X)
    assert np.allclose(g, w3 * np.tanh(w2 * np.tanh(w1 * X[:, 0])) + b3, rtol=1e-14)
    assert p["W1"].shape == (64, 5)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    theta = _theta(rng)
    X = rng.standard_normal((40, 5))
    y = rng.standard_normal(40)
    L, grad = mlp.loss_and_grad(theta, X, y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 319, 320, 383, 4479, 4543, 4608]])  # every block's edges
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, y)[0] - mlp.loss_and_grad(tm, X, y)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, grad[i])


def test_planted_error_in_the_backward_pass_is_caught():
    rng = np.random.default_rng(3)
    theta = _theta(rng)
    X = rng.standard_normal((30, 5))
    y = rng.standard_normal(30)
    _, grad = mlp.loss_and_grad(theta, X, y)
    wrong = grad.copy()
    wrong[64 * 5 + 64:64 * 5 + 64 + 64 * 64] *= -1.0  # sign of the W2 block flipped
    i = 64 * 5 + 64 + 7
    h = 1e-6
    tp, tm = theta.copy(), theta.copy()
    tp[i] += h
    tm[i] -= h
    fd = (mlp.loss_and_grad(tp, X, y)[0] - mlp.loss_and_grad(tm, X, y)[0]) / (2 * h)
    assert abs(fd - grad[i]) < 1e-6 < abs(fd - wrong[i])


def test_weighted_gradient_matches_central_differences():
    """The weighted loss mean(w (g - y)^2) of the learned preconditioner's
    training: its gradient against central differences, and two special cases
    (equal weights scale the plain loss; a weight vector that selects one pair
    gives that pair's loss times n)."""
    rng = np.random.default_rng(4)
    theta = _theta(rng)
    X = rng.standard_normal((40, 5))
    y = rng.standard_normal(40)
    w = rng.uniform(0.0, 5.0, 40)
    L, grad = mlp.loss_and_grad(theta, X, y, w)
    h = 1e-6
    for i in np.concatenate([rng.choice(mlp.N_PARAMS, 40, replace=False), [0, 4479, 4608]]):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, y, w)[0] - mlp.loss_and_grad(tm, X, y, w)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, grad[i])
    L1, g1 = mlp.loss_and_grad(theta, X, y)
    L3, g3 = mlp.loss_and_grad(theta, X, y, np.full(40, 3.0))
    assert abs(L3 - 3 * L1) <= 1e-12 * L3 and np.allclose(g3, 3 * g1, rtol=1e-12, atol=1e-15)
    sel = np.zeros(40)
    sel[7] = 1.0
    g7, _, _ = mlp.forward(theta, X[7:8])
    assert abs(mlp.loss_and_grad(theta, X, y, sel)[0] * 40 - (g7[0] - y[7]) ** 2) <= 1e-12
