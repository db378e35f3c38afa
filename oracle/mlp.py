"""FP64 CPU reference of the learned exponential map (test infrastructure).

Only the tests and the benchmark's CPU leg use this module.  It states the
network, its loss and the back-propagated gradients in plain numpy float64,
independently of the CUDA kernels, and the scaled segment residuals from the
oracle's own RK4 (Eq. 3.3 integrated at step h from a g-unit tangent, Eq. 3.5).

Network: 7 -> 256 -> 256 -> 256 -> 7 with ReLU; parameters in the order
W1 [256 x 7], b1, W2 [256 x 256], b2, W3, b3, W4 [7 x 256], b4 (W row-major, out x in).
Loss: mean over the batch and the six residual outputs of the squared error, plus
lam times the mean squared error of output 6 against log(sum of the six squared
errors + 1e-6), that target being held fixed (not differentiated).

Pinned by central finite differences of the loss, straight-line and Dormand-Prince
cases of the residuals, and the far-field bound against accelerations sampled along
integrated geodesics (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

IN, OUT, WID = 7, 7, 256
SHAPES = [("W1", (WID, IN)), ("b1", (WID,)), ("W2", (WID, WID)), ("b2", (WID,)), ("W3", (WID, WID)),
          ("b3", (WID,)), ("W4", (OUT, WID)), ("b4", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    params = np.asarray(params, np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def forward(params, X):
    p = unpack(params)
    X = np.asarray(X, np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    Z3 = H2 @ p["W3"].T + p["b3"]
    H3 = np.maximum(Z3, 0.0)
    Y = H3 @ p["W4"].T + p["b4"]
    return Y, (X, Z1, H1, Z2, H2, Z3, H3)


def error_target(params, X, T):
    """log of each sample's summed squared residual error (the error head's target)."""
    Y, _ = forward(params, X)
    d = Y[:, :6] - np.asarray(T, np.float64)
    return np.log((d * d).sum(axis=1) + 1e-6)


def loss(params, X, T, lam=0.1, e=None):
    """The loss; e (the error head's target) is recomputed unless given."""
    Y, _ = forward(params, X)
    T = np.asarray(T, np.float64)
    B = Y.shape[0]
    d = Y[:, :6] - T
    se = (d * d).sum(axis=1)
    if e is None:
        e = np.log(se + 1e-6)
    return float(se.sum() / (6 * B) + lam * ((Y[:, 6] - e) ** 2).sum() / B)


def loss_and_grads(params, X, T, lam=0.1):
    """(loss, flat gradient) by back-propagation through the layers above."""
    p = unpack(params)
    Y, (X, Z1, H1, Z2, H2, Z3, H3) = forward(params, X)
    T = np.asarray(T, np.float64)
    B = Y.shape[0]
    d = Y[:, :6] - T
    se = (d * d).sum(axis=1)
    e = np.log(se + 1e-6)              # held fixed
    L = float(se.sum() / (6 * B) + lam * ((Y[:, 6] - e) ** 2).sum() / B)
    dY = np.zeros_like(Y)
    dY[:, :6] = 2.0 * d / (6 * B)
    dY[:, 6] = 2.0 * lam * (Y[:, 6] - e) / B
    g = {}
    g["W4"] = dY.T @ H3
    g["b4"] = dY.sum(axis=0)
    dZ3 = (dY @ p["W4"]) * (Z3 > 0)
    g["W3"] = dZ3.T @ H2
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ p["W3"]) * (Z2 > 0)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return L, pack(g)


def far_field_bound(center, amplitude, sigma, cutoff, x, s):
    """Upper bound on |x''| (Eq. 5.4) along every path of Euclidean length <= s from x,
    for a g-unit tangent, over isotropic bumps (Eq. 6.1) truncated at cutoff sigma.

    |x''| = |v^T Hess f v| t / (1 + t^2), t = |grad f|, |v| <= 1 (g >= I), and
    t / (1 + t^2) <= min(t, 1/2).  For one bump at distance r, with u = r^2 / sigma^2:
    |grad f_k| = |a| q r e^{-u/2}, ||Hess f_k|| <= |a| q (1 + u) e^{-u/2}; both decrease
    in r for u >= 1, so each is taken at u = max(rho^2 q, 1), rho = max(0, |x - c| - s).
    Bumps whose support the path cannot reach (rho >= cutoff sigma) are left out.
    """
    c = np.asarray(center, np.float64).reshape(-1, 3)
    a = np.abs(np.asarray(amplitude, np.float64).reshape(-1))
    sg = np.asarray(sigma, np.float64).reshape(-1, 3)[:, 0]
    q = 1.0 / sg ** 2
    rho = np.maximum(np.linalg.norm(np.asarray(x, np.float64) - c, axis=1) - s, 0.0)
    reach = a > 0
    if cutoff > 0:
        reach &= rho < cutoff * sg
    u = np.maximum(q * rho ** 2, 1.0)
    e = a * q * np.exp(-u / 2)
    Gb = (e * np.sqrt(u / q))[reach].sum()
    Hb = (e * (1 + u))[reach].sum()
    return float(Hb * min(Gb, 0.5))


def segment_residuals(metric, X, box, s_max, h):
    """Scaled residuals (r_x, r_v) of the segments encoded in X, from the oracle's FP64 RK4."""
    from . import RK4, inner, integrate
    X = np.asarray(X, np.float64)
    out = np.zeros((X.shape[0], 6))
    for i, row in enumerate(X):
        x = row[:3] * box
        d = row[3:6]
        s = row[6] * s_max
        n = int(round(s / h))
        v = d / np.sqrt(inner(metric, x, d, d))
        xs, vs = integrate(metric, RK4, h, n, x, v)
        s_eff = n * h
        out[i, :3] = (xs[-1] - x - s_eff * v) / s_eff ** 2
        out[i, 3:] = (vs[-1] - v) / s_eff
    return out
