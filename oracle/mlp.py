"""Plain FP64 reference of the learned Davidson preconditioner's network.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/ may use it.  The
paper has no learned part; this restates the network the library trains:
g(x) = W3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 with x in R^5, 64 hidden units
per layer, and the gradient of the (weighted) mean squared error of g against
targets y.
Parameters are one flat vector in the order W1 (64 x 5, row-major), b1 (64),
W2 (64 x 64), b2 (64), W3 (64), b3 (1).

Pins (tests/test_oracle_mlp.py): the gradient against central finite
differences of the loss; special cases (zero weights give the constant b3;
a single hidden unit reduces to a closed form)."""
import numpy as np

N_IN, N_HID = 5, 64
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)), ("W3", (N_HID,)),
         ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    """Flat parameter vector -> dict of arrays (views)."""
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def forward(theta, X):
    """g for every row of X (n x 5); returns g (n,) and the hidden activations."""
    p = unpack(theta)
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    g = h2 @ p["W3"] + p["b3"][0]
    return g, h1, h2


def loss_and_grad(theta, X, y, w=None):
    """L = mean(w (g - y)^2) (w = 1 when None) and dL/dtheta (flat), by the
    chain rule layer by layer."""
    p = unpack(theta)
    g, h1, h2 = forward(theta, X)
    n = X.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    e = g - y
    L = float(np.mean(w * e * e))
    dg = 2.0 * w * e / n                   # dL/dg
    gW3 = h2.T @ dg
    gb3 = np.array([dg.sum()])
    dz2 = np.outer(dg, p["W3"]) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 * h1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
