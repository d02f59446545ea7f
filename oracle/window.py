"""FP64 reference of the windowed cost and its gradients.  Test
infrastructure only.

Over a window of n frames x_1 .. x_n (rows of X, each of m entries) with
coefficients y_1 .. y_n (columns of Y, k x n) and per-entry weights W (n x m),
the cost of Eq. (spcacost) with the weighted norm of Eq. (weightedLPnorm) summed
over the window is

    F(U, Y, mu) = sum_t sum_e W_te ((x_te - u_e^T y_t)^2 + mu)^(p/2).

With r_te = x_te - u_e^T y_t and eta_te = -p W_te r_te (r_te^2 + mu)^(p/2 - 1)
(the per-frame eta of Section 3.3, whose product with y_t is the gradient in U
and with U^T the gradient in y), the gradients are

    dF/dU = H Y^T,  dF/dY = U^T H,  H = [eta_te] (m x n),
    dF/dmu = sum_t sum_e W_te (p/2) (r_te^2 + mu)^(p/2 - 1).

This is the definition written out; the tests pin it to finite differences,
to the per-frame C oracle (n = 1), to the p = 2 closed form and to the
invariance F(U Q, Q^T Y) = F(U, Y) for orthogonal Q.
"""

from __future__ import annotations

import numpy as np


def expand_weights(labels, channels: int, omega: float) -> np.ndarray:
    """Per-entry weights (n x m) from per-pixel labels (n x P): omega where the
    label is set, 1 elsewhere, the same for every channel of a pixel (the
    weighting of Eq. (pixelweighting) and the colour rule of Section 3.4)."""
    lab = np.asarray(labels) != 0
    w = np.where(lab, omega, 1.0)
    return np.tile(w, (1, channels))


def window_cost_grad(U, Y, X, W, p: float, mu: float):
    """(F, dF/dU (m x k), dF/dY (k x n), dF/dmu) in FP64."""
    U = np.asarray(U, np.float64)
    Y = np.asarray(Y, np.float64)
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    R = X.T - U @ Y                        # m x n
    Z = R * R + mu
    F = float(np.sum(W.T * Z ** (0.5 * p)))
    H = -p * W.T * R * Z ** (0.5 * p - 1.0)
    dU = H @ Y.T
    dY = U.T @ H
    dmu = float(np.sum(W.T * (0.5 * p) * Z ** (0.5 * p - 1.0)))
    return F, dU, dY, dmu


def grassmann_window_step(U, dU, t: float):
    """One step of U along the window gradient: the projection
    G = (I - U U^T) dU of Eq. (gproject), V = U - t G, and the Cholesky-QR
    retraction V R^{-1} with V^T V = R^T R (FP64)."""
    U = np.asarray(U, np.float64)
    dU = np.asarray(dU, np.float64)
    G = dU - U @ (U.T @ dU)
    V = U - t * G
    R = np.linalg.cholesky(V.T @ V).T
    return np.linalg.solve(R.T, V.T).T
