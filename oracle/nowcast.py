"""TEST INFRASTRUCTURE ONLY -- float64 oracle of the nowcasting aggregators.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; the CUDA path never does.

The paper extrapolates wind from a context of past measurements with a
kernel-weighted average (Eq. GKA, Sec. 3.2) and truncates the context to the
few points that contribute most, i.e. the k nearest neighbours.  The
aggregators written here are the readings used by this project:

* features: for neighbour j of query q, the scaled offsets
  (sqrt(sx)(x_j-x_q), sqrt(sy)(y_j-y_q), sqrt(sz)(z_j-z_q), sqrt(st)(t_j-t_q))
  and the neighbour's measured wind (u_j, v_j); six channels per neighbour in
  neighbour-rank order, standardised channel-wise with (mean, std), zero for
  a missing neighbour.
* IDW: s_hat = sum_j w_j s_j / sum_j w_j with w_j = 1 / (d2_j + eps) over the
  valid neighbours; NaN when the context is empty.
* MLP: Z = X W1 + b1, H = GELU(Z) (erf form), Y = H W2 + b2, mean squared
  error over the B x 2 outputs, and its exact gradient.
* AdamW: Adam's moment estimates with bias correction and decoupled weight
  decay (w <- w - lr * (m_hat / (sqrt(v_hat) + eps) + wd * w)).
* GKA (Eq. GKA, Sec. 3.2): s_hat = sum_k w_k s_k / sum_k w_k over the valid
  neighbours with w_k = exp(-(s_xy ((x - x_k)^2 + (y - y_k)^2)
  + s_z (z - z_k)^2 + s_t (t - t_k)^2)); the parameters are theta = log(s)
  (s_xy, s_z, s_t > 0), trained with Adam on the same mean squared error.
* window average (Sec. 4.1, Table 2 "Hour Average"): the mean wind of every
  point measured in [t_q - before_lo, t_q - before_hi], closed at both ends
  as the paper writes [t - 1h30; t - 30min]; NaN for an empty window; the
  day average is the same mean over every point.
* GKA-MLP (Sec. 3.2: the scales as a function of the location): per query
  theta(q) = tanh(u W1 + b1) W2 + b2 with u = (q_xyz - lo) / (hi - lo) the
  location normalised by the points' bounding box, then GKA with
  s = exp(theta(q)); trained end to end with Adam.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_FEAT = 6


def features(pts, wind, queries, idx, sigma, mean=None, std=None):
    """float64 features [m, k, 6] (see module doc)."""
    pts = np.asarray(pts, dtype=np.float32)
    wind = np.asarray(wind, dtype=np.float32)
    queries = np.asarray(queries, dtype=np.float32)
    idx = np.asarray(idx)
    m, k = idx.shape
    sq = np.sqrt(np.asarray(sigma, dtype=np.float64))
    out = np.zeros((m, k, N_FEAT), dtype=np.float64)
    valid = idx >= 0
    j = np.where(valid, idx, 0)
    nb = pts[j].astype(np.float64)
    q = queries.astype(np.float64)[:, None, :]
    off = (nb - q) * sq[None, None, :]
    out[..., 0:4] = off
    out[..., 4:6] = wind[j].astype(np.float64)
    if mean is not None:
        out = (out - np.asarray(mean, dtype=np.float64)) / np.asarray(std, dtype=np.float64)
    out[~valid] = 0.0
    return out


def idw(d2, idx, wind, eps: float = 1e-6):
    """Inverse-distance-weighted average of the neighbours' wind [m, 2]."""
    d2 = np.asarray(d2, dtype=np.float64)
    idx = np.asarray(idx)
    wind = np.asarray(wind, dtype=np.float64)
    valid = idx >= 0
    w = np.where(valid, 1.0 / (np.where(valid, d2, 0.0) + eps), 0.0)
    s = wind[np.where(valid, idx, 0)]
    num = (w[..., None] * s).sum(axis=1)
    den = w.sum(axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / den[:, None]


def window_average(pts, wind, queries, before_lo: float = 5400.0, before_hi: float = 1800.0,
                   chunk: int = 256):
    """Mean wind [m, 2] (float64) of the points j with
    t_q - before_lo <= t_j <= t_q - before_hi, compared in float64 on the
    float32 times; a plain masked mean over all points for every query."""
    t = np.asarray(pts, dtype=np.float32)[:, 3].astype(np.float64)
    w = np.asarray(wind, dtype=np.float32).astype(np.float64)
    tq = np.asarray(queries, dtype=np.float32)[:, 3].astype(np.float64)
    out = np.full((tq.shape[0], 2), np.nan)
    for a in range(0, tq.shape[0], chunk):
        q = tq[a:a + chunk, None]
        mask = (t[None, :] >= q - before_lo) & (t[None, :] <= q - before_hi)
        cnt = mask.sum(axis=1)
        s = mask.astype(np.float64) @ w
        ok = cnt > 0
        out[a:a + chunk][ok] = s[ok] / cnt[ok, None]
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def mlp_forward(X, W1, b1, W2, b2):
    X = np.asarray(X, dtype=np.float64)
    Z = X @ np.asarray(W1, np.float64) + np.asarray(b1, np.float64)
    H = gelu(Z)
    Y = H @ np.asarray(W2, np.float64) + np.asarray(b2, np.float64)
    return Z, H, Y


def mse(Y, T) -> float:
    Y = np.asarray(Y, np.float64)
    T = np.asarray(T, np.float64)
    return float(np.mean((Y - T) ** 2))


def mlp_grads(X, T, W1, b1, W2, b2):
    """Loss and exact gradients of mean((Y - T)^2)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    Z, H, Y = mlp_forward(X, W1, b1, W2, b2)
    loss = float(np.mean((Y - T) ** 2))
    dY = 2.0 * (Y - T) / Y.size
    dW2 = H.T @ dY
    db2 = dY.sum(axis=0)
    dH = dY @ np.asarray(W2, np.float64).T
    dZ = dH * gelu_grad(Z)
    dW1 = X.T @ dZ
    db1 = dZ.sum(axis=0)
    return loss, dict(W1=dW1, b1=db1, W2=dW2, b2=db2)


def adamw_step(w, g, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-2):
    """One AdamW step (t counts from 1); returns new (w, m, v)."""
    w = np.asarray(w, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    w = w - lr * (mhat / (np.sqrt(vhat) + eps) + wd * w)
    return w, m, v


def gka_forward(pts, wind, queries, idx, theta):
    """GKA estimate [m, 2] (float64) and the per-neighbour weights [m, k];
    theta is [3] (one set of scales) or [m, 3] (per query).

    The exponent is evaluated relative to its smallest value over the
    context (the common factor cancels in the ratio); NaN for an empty
    context."""
    pts = np.asarray(pts, dtype=np.float32).astype(np.float64)
    wind = np.asarray(wind, dtype=np.float32).astype(np.float64)
    q = np.asarray(queries, dtype=np.float32).astype(np.float64)
    idx = np.asarray(idx)
    sig = np.exp(np.asarray(theta, dtype=np.float64))
    if sig.ndim == 1:
        sig = np.broadcast_to(sig, (q.shape[0], 3))
    sxy, sz, st = sig[:, 0:1], sig[:, 1:2], sig[:, 2:3]
    valid = idx >= 0
    j = np.where(valid, idx, 0)
    d = pts[j] - q[:, None, :]
    e = sxy * (d[..., 0] ** 2 + d[..., 1] ** 2) + sz * d[..., 2] ** 2 + st * d[..., 3] ** 2
    e = np.where(valid, e, np.inf)
    emin = np.min(e, axis=1, keepdims=True)
    w = np.where(valid, np.exp(-(e - np.where(np.isinf(emin), 0.0, emin))), 0.0)
    W = w.sum(axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        out = (w[..., None] * wind[j]).sum(axis=1) / W[:, None]
    return out, w


def gka_loss_grad(pts, wind, rows, idx, theta):
    """Self-query GKA over the dataset rows `rows` (query = the point, target
    = its wind): (loss = mean over B x 2 of (s_hat - s)^2, dloss/dtheta [3])."""
    pts = np.asarray(pts, dtype=np.float32)
    wind64 = np.asarray(wind, dtype=np.float32).astype(np.float64)
    rows = np.asarray(rows)
    idx = np.asarray(idx)[rows]
    q = pts[rows]
    pred, w = gka_forward(pts, wind, q, idx, theta)
    t = wind64[rows]
    err = pred - t
    B = rows.shape[0]
    loss = float((err ** 2).sum() / (2 * B))
    p64 = pts.astype(np.float64)
    valid = idx >= 0
    j = np.where(valid, idx, 0)
    d = p64[j] - p64[rows][:, None, :]
    sq = [d[..., 0] ** 2 + d[..., 1] ** 2, d[..., 2] ** 2, d[..., 3] ** 2]
    W = w.sum(axis=1)
    dev = wind64[j] - pred[:, None, :]  # s_k - s_hat
    sig = np.exp(np.asarray(theta, dtype=np.float64))
    g = np.zeros(3)
    for f in range(3):
        # d s_hat / d s_f = -sum_k w_k D_kf (s_k - s_hat) / W
        ds = -(w[..., None] * sq[f][..., None] * dev).sum(axis=1) / W[:, None]
        g[f] = sig[f] * (err * ds).sum() / B  # d/dtheta = s_f d/ds_f; d loss / d s_hat = err / B
    return loss, g


def gkamlp_unflatten(params, hidden: int):
    """Flat layout W1 [3][H] | b1 [H] | W2 [H][3] | b2 [3] -> arrays."""
    p = np.asarray(params, dtype=np.float64)
    H = hidden
    o = 0
    W1 = p[o:o + 3 * H].reshape(3, H); o += 3 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + 3 * H].reshape(H, 3); o += 3 * H
    b2 = p[o:o + 3]
    return W1, b1, W2, b2


def gkamlp_theta(queries, params, hidden: int, lo, hi):
    """Per-query log-scales [m, 3], hidden activations [m, H] and u [m, 3]."""
    W1, b1, W2, b2 = gkamlp_unflatten(params, hidden)
    q = np.asarray(queries, dtype=np.float32).astype(np.float64)
    lo = np.asarray(lo, dtype=np.float32).astype(np.float64)[:3]
    hi = np.asarray(hi, dtype=np.float32).astype(np.float64)[:3]
    u = (q[:, :3] - lo) / np.where(hi > lo, hi - lo, 1.0)
    h = np.tanh(u @ W1 + b1)
    return h @ W2 + b2, h, u


def gkamlp_forward(pts, wind, queries, idx, params, hidden: int, lo, hi):
    theta, _, _ = gkamlp_theta(queries, params, hidden, lo, hi)
    return gka_forward(pts, wind, queries, idx, theta)[0]


def gkamlp_loss_grad(pts, wind, rows, idx, params, hidden: int, lo, hi):
    """Self-query GKA-MLP on dataset rows: (loss, gradient in the flat layout)."""
    pts = np.asarray(pts, dtype=np.float32)
    wind64 = np.asarray(wind, dtype=np.float32).astype(np.float64)
    rows = np.asarray(rows)
    idx = np.asarray(idx)[rows]
    q = pts[rows]
    theta, h, u = gkamlp_theta(q, params, hidden, lo, hi)
    pred, w = gka_forward(pts, wind, q, idx, theta)
    t = wind64[rows]
    err = pred - t
    B = rows.shape[0]
    loss = float((err ** 2).sum() / (2 * B))
    p64 = pts.astype(np.float64)
    valid = idx >= 0
    j = np.where(valid, idx, 0)
    d = p64[j] - p64[rows][:, None, :]
    sq = [d[..., 0] ** 2 + d[..., 1] ** 2, d[..., 2] ** 2, d[..., 3] ** 2]
    W = w.sum(axis=1)
    dev = wind64[j] - pred[:, None, :]
    sig = np.exp(theta)
    dth = np.zeros_like(theta)  # d loss / d theta(q)
    for f in range(3):
        ds = -(w[..., None] * sq[f][..., None] * dev).sum(axis=1) / W[:, None]
        dth[:, f] = sig[:, f] * (err * ds).sum(axis=1) / B
    W1, b1, W2, b2 = gkamlp_unflatten(params, hidden)
    gW2 = h.T @ dth
    gb2 = dth.sum(axis=0)
    da = (dth @ W2.T) * (1.0 - h ** 2)
    gW1 = u.T @ da
    gb1 = da.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])
