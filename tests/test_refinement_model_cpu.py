"""The FP64 residual correction of the mixed-precision Davidson (the library's
`refine` option), modelled in numpy on the CPU: a reading of the paper's
FP64 Davidson for an operator applied with a relative error of ~1e-5.

The model follows the library's outer loop: an inner eigensolver on the
noisy operator runs to its noise floor; the accurate W = H X and the FP64
residual are formed; the next inner solve runs on the projected operator
H_c = P H~ P + W X^T + X W^T - X C X^T (P = I - X X^T, C = sym(X^T W)),
which equals H on X in both directions, so its lowest Ritz vector corrects
X.  Checked: the identity H_c X = H X and X^T H_c = X^T H, and that the
outer loop reaches an FP64 residual far below the noise floor, with the
eigenvalue of numpy's eigh."""
import numpy as np


def _noisy(H, eps, rng):
    """A symmetric operator whose products carry a relative error eps."""
    E = rng.standard_normal(H.shape)
    E = 0.5 * (E + E.T)
    E *= eps * np.linalg.norm(H, 2) / np.linalg.norm(E, 2)
    return H + E


def _lowest(A, x0, iters):
    """Inner solver: a few steps of inverse-free Lanczos (lowest Ritz pair of a
    Krylov space grown from x0), enough to reach the noise floor of A."""
    n = A.shape[0]
    V = np.zeros((n, iters))
    v = x0 / np.linalg.norm(x0)
    for j in range(iters):
        for _ in range(2):
            v = v - V[:, :j] @ (V[:, :j].T @ v)
        v /= np.linalg.norm(v)
        V[:, j] = v
        v = A @ v
    T = V.T @ A @ V
    w, U = np.linalg.eigh(0.5 * (T + T.T))
    x = V @ U[:, 0]
    return w[0], x / np.linalg.norm(x)


def _projected(Hn, H, X):
    P = np.eye(H.shape[0]) - X @ X.T
    W = H @ X
    C = 0.5 * (X.T @ W + W.T @ X)
    return P @ Hn @ P + W @ X.T + X @ W.T - X @ C @ X.T


def test_projected_operator_equals_h_on_x():
    rng = np.random.default_rng(3)
    n = 60
    H = rng.standard_normal((n, n))
    H = 0.5 * (H + H.T)
    Hn = _noisy(H, 1e-5, rng)
    X = np.linalg.qr(rng.standard_normal((n, 2)))[0]
    Hc = _projected(Hn, H, X)
    assert np.abs(Hc @ X - H @ X).max() < 1e-12
    assert np.abs(X.T @ Hc - X.T @ H).max() < 1e-12
    assert np.abs(Hc - Hc.T).max() < 1e-12


def test_residual_correction_reaches_fp64_accuracy():
    rng = np.random.default_rng(5)
    n = 120
    # a spectrum with a gap above the lowest eigenvalue (as at a DMRG bond)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    lam = np.concatenate([[-3.0], np.linspace(-2.0, 4.0, n - 1)])
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    Hn = _noisy(H, 1e-5, rng)
    e_ref = np.linalg.eigvalsh(H)[0]
    # plain solve on the noisy operator: stops at its floor
    th, x = _lowest(Hn, rng.standard_normal(n), 40)
    r_plain = np.linalg.norm(H @ x - (x @ H @ x) * x)
    assert r_plain > 1e-7
    # outer FP64 residual correction
    X = x[:, None]
    res = []
    for _ in range(8):
        w = H @ X[:, 0]
        rq = X[:, 0] @ w
        res.append(np.linalg.norm(w - rq * X[:, 0]))
        if res[-1] < 1e-11:
            break
        Hc = _projected(Hn, H, X)
        _, x = _lowest(Hc, X[:, 0] + 1e-3 * rng.standard_normal(n), 40)
        X = x[:, None] * np.sign(x @ X[:, 0])
    rq = X[:, 0] @ H @ X[:, 0]
    print(f"plain residual {r_plain:.2e}; corrected residuals {['%.1e' % r for r in res]}; "
          f"|E - eigh| = {abs(rq - e_ref):.2e}")
    assert res[-1] < 1e-10
    assert abs(rq - e_ref) < 1e-12
