"""Pins of the windowed cost and gradient oracle."""

import numpy as np
import pytest

import oracle
from oracle import window as wo


def _problem(m=60, k=3, n=5, seed=0, p=0.5, mu=0.05):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    Y = rng.standard_normal((k, n))
    X = (U @ Y).T + 0.1 * rng.standard_normal((n, m))
    W = np.where(rng.random((n, m)) < 0.1, 0.2, 1.0)
    return U, Y, X, W, p, mu


def test_gradients_against_central_differences():
    U, Y, X, W, p, mu = _problem()
    F, dU, dY, dmu = wo.window_cost_grad(U, Y, X, W, p, mu)
    rng = np.random.default_rng(1)
    h = 1e-6
    for A, G, name in ((U, dU, "U"), (Y, dY, "Y")):
        V = rng.standard_normal(A.shape)
        Ap, Am = A + h * V, A - h * V
        args_p = (Ap, Y) if name == "U" else (U, Ap)
        args_m = (Am, Y) if name == "U" else (U, Am)
        fd = (wo.window_cost_grad(*args_p, X, W, p, mu)[0] - wo.window_cost_grad(*args_m, X, W, p, mu)[0]) / (2 * h)
        assert fd == pytest.approx(float(np.sum(G * V)), rel=1e-6)
    fd = (wo.window_cost_grad(U, Y, X, W, p, mu + h)[0] - wo.window_cost_grad(U, Y, X, W, p, mu - h)[0]) / (2 * h)
    assert fd == pytest.approx(dmu, rel=1e-6)


def test_single_frame_matches_the_per_frame_oracle():
    # n = 1: the window cost and gradients are the per-frame ones of the C oracle
    width, height, C, k = 7, 5, 2, 3
    prm = oracle.params(width, height, C, k, p=0.3, mu=0.07, omega=0.25)
    m, P = C * width * height, width * height
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    y = rng.standard_normal(k)
    x = rng.standard_normal(m)
    labels = (rng.random(P) < 0.3).astype(np.uint8)
    w_pix = oracle.weights(prm, labels)
    W = wo.expand_weights(labels[None, :], C, 0.25)
    F, dU, dY, dmu = wo.window_cost_grad(U, y[:, None], x[None, :], W, 0.3, 0.07)
    assert F == pytest.approx(oracle.cost(prm, U, y, x, w_pix), rel=1e-13)
    eta = oracle.eta(prm, oracle.residual(U, y, x), w_pix)
    np.testing.assert_allclose(dU, oracle.grad_U(eta, y), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(dY[:, 0], oracle.ut(U, eta), rtol=1e-12, atol=1e-15)


def test_p2_closed_form():
    U, Y, X, W, _, mu = _problem(p=2.0)
    F, dU, dY, dmu = wo.window_cost_grad(U, Y, X, W, 2.0, mu)
    R = X.T - U @ Y
    assert F == pytest.approx(float(np.sum(W.T * (R * R + mu))), rel=1e-13)
    np.testing.assert_allclose(dU, -2.0 * (W.T * R) @ Y.T, rtol=1e-12)
    np.testing.assert_allclose(dY, -2.0 * U.T @ (W.T * R), rtol=1e-12)
    assert dmu == pytest.approx(float(W.sum()), rel=1e-13)


def test_rotation_invariance():
    U, Y, X, W, p, mu = _problem(seed=3)
    Q, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((3, 3)))
    F, dU, dY, dmu = wo.window_cost_grad(U, Y, X, W, p, mu)
    F2, dU2, dY2, dmu2 = wo.window_cost_grad(U @ Q, Q.T @ Y, X, W, p, mu)
    assert F2 == pytest.approx(F, rel=1e-13)
    np.testing.assert_allclose(dU2, dU @ Q, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(dY2, Q.T @ dY, rtol=1e-10, atol=1e-13)
    assert dmu2 == pytest.approx(dmu, rel=1e-13)


def test_window_step_is_the_unique_qr_and_descends():
    U, Y, X, W, p, mu = _problem(m=80, k=4, n=6, seed=5)
    F, dU, dY, dmu = wo.window_cost_grad(U, Y, X, W, p, mu)
    Q = wo.grassmann_window_step(U, dU, 1e-3)
    V = U - 1e-3 * (dU - U @ (U.T @ dU))
    q, r = np.linalg.qr(V)
    q = q * np.sign(np.diag(r))      # positive diagonal: the unique QR
    np.testing.assert_allclose(Q, q, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-12)
    np.testing.assert_allclose(wo.grassmann_window_step(U, dU, 0.0), U, atol=1e-12)
    F2 = wo.window_cost_grad(Q, Y, X, W, p, mu)[0]
    assert F2 < F
