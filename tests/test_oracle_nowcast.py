"""Pins of the nowcast oracle: GELU against the standard normal CDF, the
MLP forward on a hand-worked 2-2-2 network, the MLP gradient against central
finite differences, AdamW against its closed form under a constant
gradient, IDW special cases, a hand-worked feature row, GKA closed forms and
the GKA-MLP scales on a hand-worked one-unit network."""
import math

import numpy as np
import pytest

from oracle import nowcast as nc


def test_gelu_known_values():
    # GELU(z) = z * Phi(z); standard normal table values Phi(1) =
    # 0.841344746068543, Phi(-1) = 0.158655253931457, Phi(6) = 1 - 9.8659e-10
    z = np.array([0.0, 1.0, -1.0, 6.0])
    np.testing.assert_allclose(nc.gelu(z), [0.0, 0.841344746068543, -0.158655253931457,
                                            6.0 * (1.0 - 9.8659e-10)], rtol=1e-12, atol=1e-12)


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    B, din, dh = 7, 12, 9
    X = rng.normal(size=(B, din))
    T = rng.normal(size=(B, 2))
    P = dict(W1=rng.normal(size=(din, dh)) * 0.4, b1=rng.normal(size=dh) * 0.1,
             W2=rng.normal(size=(dh, 2)) * 0.4, b2=rng.normal(size=2) * 0.1)
    loss, g = nc.mlp_grads(X, T, **P)
    h = 1e-6
    for name in P:
        flat = P[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 11)):
            old = flat[i]
            flat[i] = old + h
            lp = nc.mse(nc.mlp_forward(X, **P)[2], T)
            flat[i] = old - h
            lm = nc.mse(nc.mlp_forward(X, **P)[2], T)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert g[name].reshape(-1)[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adamw_constant_gradient_closed_form():
    # With a constant gradient g, m_hat = g and v_hat = g^2 at every step, so
    # w_{t+1} = (1 - lr wd) w_t - lr g / (|g| + eps): a geometric recursion
    # with the closed form w_t = c^t w_0 - lr s (1 - c^t) / (1 - c).
    lr, wd, eps = 1e-2, 0.1, 1e-8
    g = np.array([0.5, -2.0, 3e-4])
    w0 = np.array([1.0, -1.0, 0.25])
    w, m, v = w0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 26):
        w, m, v = nc.adamw_step(w, g, m, v, t, lr=lr, wd=wd, eps=eps)
    c = 1.0 - lr * wd
    s = g / (np.abs(g) + eps)
    closed = c ** 25 * w0 - lr * s * (1 - c ** 25) / (1 - c)
    np.testing.assert_allclose(w, closed, rtol=1e-9)


def test_idw_special_cases():
    wind = np.array([[3.0, 4.0], [3.0, 4.0], [3.0, 4.0], [-1.0, 2.0]])
    # constant field -> that constant
    out = nc.idw(np.array([[1.0, 2.0, 5.0]]), np.array([[0, 1, 2]]), wind)
    np.testing.assert_allclose(out, [[3.0, 4.0]])
    # a single neighbour -> its value; missing neighbours are ignored
    out = nc.idw(np.array([[7.0, np.inf]]), np.array([[3, -1]]), wind)
    np.testing.assert_allclose(out, [[-1.0, 2.0]])
    # two neighbours at d2 = 1 and 3 (eps = 0): weights 1 and 1/3
    out = nc.idw(np.array([[1.0, 3.0]]), np.array([[0, 3]]), wind, eps=0.0)
    np.testing.assert_allclose(out, [[(3.0 - 1.0 / 3) / (4.0 / 3), (4.0 + 2.0 / 3) / (4.0 / 3)]])
    # permutation invariance
    a = nc.idw(np.array([[1.0, 2.0, 4.0]]), np.array([[0, 3, 1]]), wind)
    b = nc.idw(np.array([[4.0, 1.0, 2.0]]), np.array([[1, 0, 3]]), wind)
    np.testing.assert_allclose(a, b)
    # empty context -> NaN
    assert np.isnan(nc.idw(np.array([[np.inf]]), np.array([[-1]]), wind)).all()


def test_features_hand_row():
    pts = np.array([[10.0, 20.0, 9.0, 100.0], [12.0, 17.0, 10.0, 60.0]], np.float32)
    wind = np.array([[1.0, 2.0], [5.0, -3.0]], np.float32)
    q = np.array([[10.0, 20.0, 9.0, 100.0]], np.float32)
    f = nc.features(pts, wind, q, np.array([[1, -1]]), (1.0, 4.0, 9.0, 0.01))
    # offsets scaled by sqrt(sigma) = (1, 2, 3, 0.1): (2, -6, 3, -4), wind (5, -3)
    np.testing.assert_allclose(f[0, 0], [2.0, -6.0, 3.0, -4.0, 5.0, -3.0], rtol=1e-7)
    np.testing.assert_array_equal(f[0, 1], np.zeros(6))
    g = nc.features(pts, wind, q, np.array([[1, -1]]), (1.0, 4.0, 9.0, 0.01),
                    mean=np.ones(6), std=np.full(6, 2.0))
    np.testing.assert_allclose(g[0, 0], [0.5, -3.5, 1.0, -2.5, 2.0, -2.0], rtol=1e-7)
    np.testing.assert_array_equal(g[0, 1], np.zeros(6))


def _gka_case(seed=3, n=120, k=6):
    rng = np.random.default_rng(seed)
    pts = np.column_stack([rng.uniform(0, 5, n), rng.uniform(0, 5, n), rng.uniform(8, 11, n),
                           rng.uniform(0, 300, n)]).astype(np.float32)
    wind = rng.normal(0, 10, size=(n, 2)).astype(np.float32)
    idx = np.array([rng.choice(n, k, replace=False) for _ in range(n)], dtype=np.int32)
    return pts, wind, idx


def test_gka_equal_weights_give_the_plain_average():
    # every neighbour at the same offset pattern -> equal weights
    pts = np.array([[0, 0, 10, 100], [1, 0, 10, 90], [-1, 0, 10, 90], [0, 1, 10, 90], [0, -1, 10, 90]],
                   np.float32)
    wind = np.array([[0, 0], [1, 2], [3, 4], [5, 6], [7, 8]], np.float32)
    idx = np.array([[1, 2, 3, 4]], np.int32)
    out, w = nc.gka_forward(pts, wind, pts[:1], idx, np.log([0.7, 2.0, 0.01]))
    np.testing.assert_allclose(w, 1.0)
    np.testing.assert_allclose(out, [[4.0, 5.0]], rtol=1e-12)


def test_gka_two_neighbours_closed_form():
    # two neighbours: s_hat = (s1 + r s2) / (1 + r), r = exp(-(e2 - e1))
    pts = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 2, 1, -3]], np.float32)
    wind = np.array([[0, 0], [2, -1], [6, 3]], np.float32)
    th = np.log([0.5, 3.0, 0.2])
    out, _ = nc.gka_forward(pts, wind, pts[:1], np.array([[1, 2]], np.int32), th)
    e1 = 0.5 * 1.0
    e2 = 0.5 * 4.0 + 3.0 * 1.0 + 0.2 * 9.0
    r = math.exp(-(e2 - e1))
    np.testing.assert_allclose(out[0], (np.array([2, -1]) + r * np.array([6, 3])) / (1 + r), rtol=1e-12)


def test_gka_large_scale_tends_to_the_nearest_neighbour_and_ignores_missing():
    pts, wind, idx = _gka_case()
    idx[:, -1] = -1  # a missing neighbour changes nothing
    out, _ = nc.gka_forward(pts, wind, pts, idx, np.log([1e4, 1e4, 1e4]))
    d = pts[np.where(idx >= 0, idx, 0)].astype(np.float64) - pts[:, None, :].astype(np.float64)
    e = 1e4 * (d ** 2).sum(axis=2)
    e[idx < 0] = np.inf
    nearest = idx[np.arange(len(idx)), np.argmin(e, axis=1)]
    np.testing.assert_allclose(out, wind[nearest], rtol=1e-6, atol=1e-6)


def test_gka_gradient_matches_central_differences():
    pts, wind, idx = _gka_case(seed=8)
    rows = np.arange(0, 120, 3)
    th = np.log([0.3, 0.8, 1e-3])
    _, g = nc.gka_loss_grad(pts, wind, rows, idx, th)
    h = 1e-6
    for f in range(3):
        tp = th.copy()
        tp[f] += h
        tm = th.copy()
        tm[f] -= h
        fd = (nc.gka_loss_grad(pts, wind, rows, idx, tp)[0] - nc.gka_loss_grad(pts, wind, rows, idx, tm)[0]) / (2 * h)
        assert abs(fd - g[f]) <= 1e-6 * max(1.0, abs(fd)), (f, fd, g[f])


def _gkamlp_params(H, seed, w2_scale=0.3):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(-1, 1, 3 * H), rng.uniform(-1, 1, H),
                           w2_scale * rng.normal(size=3 * H), np.log([0.3, 0.8, 1e-3])])


def test_gkamlp_with_zero_output_weights_is_plain_gka():
    pts, wind, idx = _gka_case(seed=5)
    H = 8
    p = _gkamlp_params(H, 1, w2_scale=0.0)
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    out = nc.gkamlp_forward(pts, wind, pts, idx, p, H, lo, hi)
    ref, _ = nc.gka_forward(pts, wind, pts, idx, np.log([0.3, 0.8, 1e-3]))
    np.testing.assert_allclose(out, ref, rtol=1e-12)


def test_gkamlp_gradient_matches_central_differences():
    pts, wind, idx = _gka_case(seed=9)
    H = 6
    p = _gkamlp_params(H, 2)
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    rows = np.arange(0, 120, 2)
    _, g = nc.gkamlp_loss_grad(pts, wind, rows, idx, p, H, lo, hi)
    h = 1e-6
    for i in range(0, p.size, 3):
        pp = p.copy()
        pp[i] += h
        pm = p.copy()
        pm[i] -= h
        fd = (nc.gkamlp_loss_grad(pts, wind, rows, idx, pp, H, lo, hi)[0]
              - nc.gkamlp_loss_grad(pts, wind, rows, idx, pm, H, lo, hi)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_forward_hand_worked_network():
    # A 2-input, 2-hidden, 2-output network worked by hand (W1 is d_in x
    # d_hidden, W2 is d_hidden x 2):
    #   W1 = [[1, -1], [0.5, 2]], b1 = [-1, -4], W2 = [[2, 1], [3, -1]],
    #   b2 = [0.1, -0.2].
    # Row x = (1, 2): Z = (1 + 1 - 1, -1 + 4 - 4) = (1, -1), so
    #   H = (Phi(1), -Phi(-1)) with the normal-table values Phi(1) =
    #   0.841344746068543, Phi(-1) = 0.158655253931457;
    #   Y = (2 Phi(1) - 3 Phi(-1) + 0.1, Phi(1) + Phi(-1) - 0.2) = (1.306723730342715, 0.8).
    # Row x = (0, -1): Z = (-0.5 - 1, -2 - 4) = (-1.5, -6), so
    #   H = (-1.5 Phi(-1.5), -6 Phi(-6)) with Phi(-1.5) = 0.0668072012688581 and
    #   Phi(-6) = 9.865876450377e-10: H = (-0.10021080190328715, -5.9195258702262e-9);
    #   Y = (-0.10042162156515191, -0.30021079598376128).
    X = np.array([[1.0, 2.0], [0.0, -1.0]])
    W1 = np.array([[1.0, -1.0], [0.5, 2.0]])
    b1 = np.array([-1.0, -4.0])
    W2 = np.array([[2.0, 1.0], [3.0, -1.0]])
    b2 = np.array([0.1, -0.2])
    Z, H, Y = nc.mlp_forward(X, W1, b1, W2, b2)
    np.testing.assert_allclose(Z, [[1.0, -1.0], [-1.5, -6.0]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(H, [[0.841344746068543, -0.158655253931457],
                                   [-0.10021080190328715, -5.9195258702262e-9]], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Y, [[1.306723730342715, 0.8],
                                   [-0.10042162156515191, -0.30021079598376128]], rtol=1e-12, atol=1e-14)


def test_gkamlp_theta_hand_worked_single_hidden_unit():
    # H = 1 hidden unit.  Bounding box lo = (0, 100, 8), hi = (10, 300, 12);
    # query (5, 150, 11) -> u = (5/10, 50/200, 3/4) = (0.5, 0.25, 0.75).
    # W1 = (2, -4, 1)^T, b1 = 0.25: pre-activation 1 - 1 + 0.75 + 0.25 = 1,
    # h = tanh(1) = 0.7615941559557649.  W2 = (1, -2, 0.5), b2 = (0.1, 0.2, -3):
    # theta = (0.1 + h, 0.2 - 2h, -3 + h/2)
    #       = (0.8615941559557649, -1.3231883119115298, -2.6192029220221176).
    params = np.array([2.0, -4.0, 1.0,   # W1 [3][1]
                       0.25,             # b1 [1]
                       1.0, -2.0, 0.5,   # W2 [1][3]
                       0.1, 0.2, -3.0])  # b2 [3]
    lo = np.array([0.0, 100.0, 8.0, 0.0], np.float32)
    hi = np.array([10.0, 300.0, 12.0, 50.0], np.float32)
    q = np.array([[5.0, 150.0, 11.0, 20.0]], np.float32)
    theta, h, u = nc.gkamlp_theta(q, params, 1, lo, hi)
    np.testing.assert_allclose(u, [[0.5, 0.25, 0.75]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(h, [[0.7615941559557649]], rtol=1e-14)
    np.testing.assert_allclose(theta, [[0.8615941559557649, -1.3231883119115298, -2.6192029220221176]],
                               rtol=1e-14)
    # the nowcast then uses s = exp(theta) in Eq. GKA: one neighbour at
    # offset (1, 0, 0, 0) and one at (0, 0, 1, 0) weigh exp(-s_xy) and
    # exp(-s_z) relative to each other
    pts = np.array([[5.0, 150.0, 11.0, 20.0], [6.0, 150.0, 11.0, 20.0], [5.0, 150.0, 12.0, 20.0]],
                   np.float32)
    wind = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], np.float32)
    out = nc.gkamlp_forward(pts, wind, q, np.array([[1, 2]], np.int32), params, 1, lo, hi)
    w1 = math.exp(-math.exp(0.8615941559557649))
    w2 = math.exp(-math.exp(-1.3231883119115298))
    np.testing.assert_allclose(out, [[w1 / (w1 + w2), w2 / (w1 + w2)]], rtol=1e-12)


def test_hour_average_hand_worked_window():
    # Hour average of Sec. 4.1: the mean of the points measured in
    # [t - 1 h 30, t - 30 min].  For a query at t = 6000 s the window is
    # [600, 4200] s, both ends included.
    t = np.array([0.0, 599.5, 600.0, 1000.0, 4200.0, 4200.5, 5000.0, 6000.0])
    u = np.array([100.0, 50.0, 1.0, 2.0, 6.0, 70.0, 80.0, 90.0])
    v = np.array([-100.0, -50.0, 4.0, 0.0, -1.0, -70.0, -80.0, -90.0])
    pts = np.column_stack([np.zeros_like(t), np.zeros_like(t), np.full_like(t, 10.0), t]).astype(np.float32)
    wind = np.column_stack([u, v]).astype(np.float32)
    q = np.array([[0.0, 0.0, 10.0, 6000.0],   # points at 600, 1000, 4200: u (1+2+6)/3, v (4+0-1)/3
                  [0.0, 0.0, 10.0, 2000.0],   # window [-3400, 200]: only t = 0
                  [0.0, 0.0, 10.0, 1000.0]],  # window [-4400, -800]: empty
                 np.float32)
    out = nc.window_average(pts, wind, q)
    np.testing.assert_allclose(out[0], [3.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(out[1], [100.0, -100.0], rtol=1e-15)
    assert np.isnan(out[2]).all()
    # the day average: every point, whatever the query time
    day = nc.window_average(pts, wind, q[:1], before_lo=np.inf, before_hi=-np.inf)
    np.testing.assert_allclose(day[0], [u.mean(), v.mean()], rtol=1e-15)
