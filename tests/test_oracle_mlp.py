"""Pins of the FP64 MLP / POD reference used to check the warm-start kernels."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    widths = [5, 7, 6, 3]
    _, n = mlp.layout(widths)
    p = rng.normal(size=n) * 0.5
    X = rng.normal(size=(4, 5))
    T = rng.normal(size=(4, 3))
    w = rng.uniform(0.5, 2.0, size=3)
    L, g = mlp.loss_grad(p, widths, X, T, w)
    h = 1e-6
    fd = np.array([(mlp.loss_grad(p + h * e, widths, X, T, w)[0] -
                    mlp.loss_grad(p - h * e, widths, X, T, w)[0]) / (2 * h) for e in np.eye(n)])
    assert np.abs(g - fd).max() < 1e-8 * max(1.0, np.abs(fd).max())


def test_single_linear_layer_is_least_squares():
    """One linear layer: the gradient is the closed form of linear least squares
    and the minimiser is the normal-equations solution."""
    rng = np.random.default_rng(1)
    widths = [4, 2]
    X = rng.normal(size=(50, 4))
    Wt = rng.normal(size=(2, 4))
    bt = rng.normal(size=2)
    T = X @ Wt.T + bt
    Xa = np.hstack([X, np.ones((50, 1))])
    sol = np.linalg.lstsq(Xa, T, rcond=None)[0]
    p = np.concatenate([sol[:4].T.ravel(), sol[4]])
    L, g = mlp.loss_grad(p, widths, X, T)
    assert L < 1e-24 and np.abs(g).max() < 1e-12
    p0 = np.zeros(10)
    L0, g0 = mlp.loss_grad(p0, widths, X, T)
    gW = -2.0 * T.T @ X / (50 * 2)
    assert np.allclose(g0[:8], gW.ravel()) and np.allclose(g0[8:], -2.0 * T.sum(0) / 100)


def test_adam_first_step_moves_by_lr_sign():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)


def test_pod_reconstructs_low_rank_snapshots():
    rng = np.random.default_rng(2)
    basis = np.linalg.qr(rng.normal(size=(200, 5)))[0]
    coef = rng.normal(size=(5, 40)) * np.array([10, 5, 2, 1, 0.5])[:, None]
    Y = basis @ coef + rng.normal(size=200)[:, None]
    mean, U, s = mlp.pod(Y, 5)
    R = U @ (U.T @ (Y - mean[:, None])) + mean[:, None]
    assert np.abs(R - Y).max() < 1e-9
    assert np.allclose(U.T @ U, np.eye(5), atol=1e-12)
    assert np.all(np.diff(s) <= 0)


def test_linear_fit_recovers_exact_maps_and_matches_lstsq():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(80, 6))
    Wt = rng.normal(size=(4, 6))
    assert np.abs(mlp.linear_fit(X, X @ Wt.T, 0.0) - Wt).max() < 1e-12
    Y = rng.normal(size=(80, 4))
    ref = np.linalg.lstsq(X, Y, rcond=None)[0].T
    assert np.abs(mlp.linear_fit(X, Y, 0.0) - ref).max() < 1e-12
    # ridge: the solution of the augmented least-squares problem [X; sqrt(c) I]
    lam = 0.1
    c = lam * np.trace(X.T @ X) / 6
    Xa = np.vstack([X, np.sqrt(c) * np.eye(6)])
    Ya = np.vstack([Y, np.zeros((6, 4))])
    ref = np.linalg.lstsq(Xa, Ya, rcond=None)[0].T
    assert np.abs(mlp.linear_fit(X, Y, lam) - ref).max() < 1e-12
