"""Double-precision reference of the learned-CDF bucketer's model and training gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The learned path is an extension of the
paper's method (the paper has no learned component), so this reference is pinned by its own
mathematics rather than by the paper: finite differences of the loss, and closed forms of the
model at its initial point.

Model (16 hidden units): with theta = [alpha(16), omega(16), c(16)],
    a = softmax(alpha),  w = exp(omega),  xn = (x - mu) / sigma,
    h_j = clamp(w_j * (xn - c_j), 0, 1),  F(x) = sum_j a_j h_j   (ramp j starts at c_j).
Loss over points (x_i, t_i): L = sum_i 0.5 * (F(x_i) - t_i)^2.
Bucket of x among nb buckets: min(nb - 1, floor(nb * F(x))) (NaN by sign: first / last).
"""

from __future__ import annotations

import numpy as np

HIDDEN = 16


def split(theta: np.ndarray):
    theta = np.asarray(theta, dtype=np.float64)
    return theta[:HIDDEN], theta[HIDDEN:2 * HIDDEN], theta[2 * HIDDEN:3 * HIDDEN]


def softmax(v: np.ndarray) -> np.ndarray:
    e = np.exp(v - v.max())
    return e / e.sum()


def forward(theta, x, mu, sigma):
    """F at each x (float64), with the hidden pre-activations z and outputs h."""
    alpha, omega, c = split(theta)
    a = softmax(alpha)
    w = np.exp(omega)
    xn = (np.asarray(x, dtype=np.float64) - mu) / sigma
    z = (xn[:, None] - c[None, :]) * w[None, :]
    h = np.clip(z, 0.0, 1.0)
    return h @ a, z, h, a, w, xn


def loss(theta, x, t, mu, sigma) -> float:
    F = forward(theta, x, mu, sigma)[0]
    return float(0.5 * np.sum((F - np.asarray(t, dtype=np.float64)) ** 2))


def loss_grad(theta, x, t, mu, sigma):
    """(loss, gradient) by the chain rule: dF/dalpha_k = a_k (h_k - F) (softmax),
    dF/domega_j = a_j [0 < z_j < 1] (xn - c_j) w_j, dF/dc_j = -a_j [0 < z_j < 1] w_j."""
    F, z, h, a, w, xn = forward(theta, x, mu, sigma)
    c = split(theta)[2]
    e = F - np.asarray(t, dtype=np.float64)
    inside = ((z > 0.0) & (z < 1.0)).astype(np.float64)
    g_alpha = (e[:, None] * a[None, :] * (h - F[:, None])).sum(axis=0)
    g_omega = (e[:, None] * a[None, :] * inside * (xn[:, None] - c[None, :]) * w[None, :]).sum(axis=0)
    g_c = -(e[:, None] * a[None, :] * inside * w[None, :]).sum(axis=0)
    return float(0.5 * np.sum(e * e)), np.concatenate([g_alpha, g_omega, g_c])


def init_theta(sorted_finite: np.ndarray, mu: float, sigma: float) -> np.ndarray:
    """Initial point: ramp j rises from 0 to 1 across the j-th sixteenth of the sorted sample."""
    x = np.asarray(sorted_finite, dtype=np.float64)
    n = x.size
    theta = np.zeros(3 * HIDDEN)
    for j in range(HIDDEN):
        q0 = (x[(n * j) // HIDDEN] - mu) / sigma
        q1 = (x[(n * (j + 1) - 1) // HIDDEN] - mu) / sigma
        width = max(q1 - q0, 1e-6)
        theta[HIDDEN + j] = -np.log(width)
        theta[2 * HIDDEN + j] = q0
    return theta


def buckets(theta, x, mu, sigma, nb: int = 4096) -> np.ndarray:
    """Bucket of each key under the model (float64 evaluation; NaNs by sign)."""
    x = np.asarray(x)
    F = forward(theta, np.where(np.isnan(x), 0.0, x), mu, sigma)[0]
    b = np.minimum(nb - 1, np.floor(nb * F)).astype(np.int64)
    nan = np.isnan(x)
    neg = np.signbit(x)
    b[nan & neg] = 0
    b[nan & ~neg] = nb - 1
    return b
