"""Parity of the nowcast kernels with the float64 oracle (features, IDW, MLP
forward, gradient, AdamW), the checkpoint round trip, and what the trained
MLP gains over the IDW fallback on held-out flights."""
import numpy as np
import pytest
import torch

import oracle
from oracle import nowcast as nc
from paper_2112_10408_gb300 import synth
from paper_2112_10408_gb300 import tnn

pytestmark = pytest.mark.gpu
SIG = synth.SIGMA_DEFAULT


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_10408_gb300 import build
    build.build()
    tnn.load_library()


def _bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_features_and_idw_match_oracle():
    wl = synth.flights(40, 60, seed=31, n_routes=4)
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 10)
    idx, d2 = tnn.tnn_knn(ix, 32, 30.0)
    wind = torch.from_numpy(wl.wind).cuda()
    mean = np.array([0.5, -1.0, 0.2, -3.0, 20.0, 5.0], np.float32)
    std = np.array([10.0, 12.0, 2.0, 4.0, 8.0, 8.0], np.float32)
    feat, idw = tnn.tnn_context_features(ix, wind, idx, d2, mean=mean, std=std)
    torch.cuda.synchronize()
    i_np, d_np = idx.cpu().numpy(), d2.cpu().numpy()
    ref = nc.features(wl.xyzt, wl.wind, wl.xyzt, i_np, SIG, mean, std).reshape(wl.n, -1)
    np.testing.assert_allclose(feat.float().cpu().numpy(), ref, rtol=1e-2, atol=1e-2)
    ref_idw = nc.idw(d_np, i_np, wl.wind)
    got = idw.cpu().numpy()
    nan = np.isnan(ref_idw)
    assert np.array_equal(np.isnan(got), nan)
    np.testing.assert_allclose(got[~nan], ref_idw[~nan], rtol=1e-5, atol=1e-5)


def _mlp_with_params(d_in, dh, seed=0):
    m = tnn.MLP(d_in, dh, seed=seed)
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.1, size=m.n_params).astype(np.float32)
    m.set_params(w)
    return m, w


def test_mlp_forward_matches_oracle():
    m, w = _mlp_with_params(192, 256)
    W1, b1, W2, b2 = m.unflatten(w.astype(np.float64))
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, size=(777, 192)).astype(np.float32)
    xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    y = m.forward(xb).cpu().numpy()
    _, _, Yr = nc.mlp_forward(_bf16_round(X), _bf16_round(W1), b1, W2, b2)
    np.testing.assert_allclose(y, Yr, rtol=2e-2, atol=2e-2 * np.abs(Yr).max())


@pytest.mark.parametrize("d_in,dh,B", [(192, 256, 60001), (96, 128, 20000), (64, 64, 3000)])
def test_mlp_inference_many_tiles(d_in, dh, B):
    """Inference over many 128-row tiles (several per CTA of the persistent
    kernel, both X buffers and both accumulators reused; a ragged last
    tile) against the oracle on every row."""
    m, w = _mlp_with_params(d_in, dh, seed=8)
    W1, b1, W2, b2 = m.unflatten(w.astype(np.float64))
    rng = np.random.default_rng(9)
    X = rng.normal(0, 1, size=(B, d_in)).astype(np.float32)
    xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    y = m.forward(xb).cpu().numpy()
    _, _, Yr = nc.mlp_forward(_bf16_round(X), _bf16_round(W1), b1, W2, b2)
    np.testing.assert_allclose(y, Yr, rtol=2e-2, atol=2e-2 * np.abs(Yr).max())
    # the same rows answered in another batch give the same values
    y2 = m.forward(xb[B // 3:]).cpu().numpy()
    np.testing.assert_array_equal(y2, y[B // 3:])


@pytest.mark.parametrize("d_in,dh", [(192, 256), (512, 512)])
def test_mlp_gradients_match_oracle(d_in, dh):
    """(192, 256) stages every K step at once; (512, 512) does not fit and
    streams the K steps through four stages."""
    m, w = _mlp_with_params(d_in, dh, seed=2)
    W1, b1, W2, b2 = m.unflatten(w.astype(np.float64))
    rng = np.random.default_rng(3)
    B = 1000
    X = rng.normal(0, 1, size=(B, d_in)).astype(np.float32)
    T = rng.normal(0, 1, size=(B, 2)).astype(np.float32)
    loss, g = m.gradients(torch.from_numpy(X).to(torch.bfloat16).cuda(), torch.from_numpy(T).cuda())
    g = g.cpu().numpy().astype(np.float64)
    lr, gr = nc.mlp_grads(_bf16_round(X), T, _bf16_round(W1), b1, W2, b2)
    assert float(loss.item()) == pytest.approx(lr, rel=2e-2)
    gW1, gb1, gW2, gb2 = m.unflatten(g)
    # element by element: BF16 operands (relative 2^-8 each) and FP32
    # accumulation over <= 1000 rows; the absolute part is 2e-2 of the
    # block's largest entry, so one wrong entry cannot hide in a norm
    for name, got in (("W1", gW1), ("b1", gb1), ("W2", gW2), ("b2", gb2)):
        ref = gr[name]
        np.testing.assert_allclose(got, ref, rtol=2e-2, atol=2e-2 * np.abs(ref).max(), err_msg=name)


def test_adamw_step_matches_oracle_update():
    m, w = _mlp_with_params(64, 64, seed=4)
    rng = np.random.default_rng(5)
    X = torch.from_numpy(rng.normal(0, 1, size=(300, 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    T = torch.from_numpy(rng.normal(0, 1, size=(300, 2)).astype(np.float32)).cuda()
    opt = tnn.AdamW(lr=3e-3, weight_decay=0.05)
    wk = w.astype(np.float64)
    mm = np.zeros_like(wk)
    vv = np.zeros_like(wk)
    for t in range(1, 4):
        _, g = m.gradients(X, T)
        g = g.cpu().numpy().astype(np.float64)
        m.train_step(X, T, opt)
        wk, mm, vv = nc.adamw_step(wk, g, mm, vv, t, lr=opt.lr, beta1=opt.beta1, beta2=opt.beta2,
                                   eps=opt.eps, wd=opt.weight_decay)
        got = m.get_params().astype(np.float64)
        np.testing.assert_allclose(got, wk, rtol=1e-5, atol=1e-7)


def test_checkpoint_round_trip(tmp_path):
    m, _ = _mlp_with_params(64, 64, seed=6)
    rng = np.random.default_rng(7)
    X = torch.from_numpy(rng.normal(0, 1, size=(128, 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    T = torch.from_numpy(rng.normal(0, 1, size=(128, 2)).astype(np.float32)).cuda()
    m.train_step(X, T, tnn.AdamW())
    p = tmp_path / "mlp.bin"
    m.save(str(p))
    m2 = tnn.MLP(64, 64, seed=99)
    m2.load(str(p))
    a = m.get_params(with_moments=True)
    b = m2.get_params(with_moments=True)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3] == b[3] == 1
    m.train_step(X, T, tnn.AdamW())
    m2.train_step(X, T, tnn.AdamW())
    np.testing.assert_array_equal(m.get_params(), m2.get_params())


def test_nowcast_entry_point_composes_the_stages():
    wl = synth.flights(30, 60, seed=41, n_routes=3)
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 10)
    wind = torch.from_numpy(wl.wind).cuda()
    uv = tnn.tnn_nowcast(ix, wind, 8, 20.0)
    idx, d2 = tnn.tnn_knn(ix, 8, 20.0)
    _, idw = tnn.tnn_context_features(ix, wind, idx, d2, want_feat=False)
    torch.testing.assert_close(uv, idw, equal_nan=True)
    m = tnn.MLP(48, 64, seed=1)
    uvm = tnn.tnn_nowcast(ix, wind, 8, 20.0, mlp=m)
    feat, _ = tnn.tnn_context_features(ix, wind, idx, d2, want_idw=False)
    torch.testing.assert_close(uvm, m.forward(feat))


def test_trained_mlp_beats_idw_on_held_out_flights():
    # Learned form at reduced size: TNN contexts (k = 32, lag 1800 s) of
    # 120,000 points, 80/20 split by flight, features standardised on the
    # training split, AdamW, batch 4096.
    wl = synth.flights(600, 200, seed=synth.SEED_LEARNED)
    k, lag = 32, 1800.0
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 20)
    idx, d2 = tnn.tnn_knn(ix, k, lag)
    wind = torch.from_numpy(wl.wind).cuda()
    full = (idx >= 0).all(dim=1).cpu().numpy()
    train, test = synth.flight_split(wl)
    tr = np.nonzero(train & full)[0]
    te = np.nonzero(test & full)[0]
    assert tr.size > 20000 and te.size > 5000
    raw, idw = tnn.tnn_context_features(ix, wind, idx, d2)
    f = raw.float()[torch.from_numpy(tr).cuda()].view(-1, k, 6)
    mean = f.mean(dim=(0, 1)).cpu().numpy()
    std = f.std(dim=(0, 1)).cpu().numpy() + 1e-6
    feat, _ = tnn.tnn_context_features(ix, wind, idx, d2, mean=mean, std=std, want_idw=False)
    y = wind
    mlp = tnn.MLP(k * 6, 256, seed=0)
    opt = tnn.AdamW(lr=1e-3, weight_decay=1e-2)
    rng = np.random.default_rng(0)
    trd = torch.from_numpy(tr).cuda()
    for epoch in range(12):
        perm = trd[torch.from_numpy(rng.permutation(tr.size)).cuda()]
        for b in range(0, perm.numel() - 4095, 4096):
            sel = perm[b:b + 4096]
            mlp.train_step(feat[sel].contiguous(), y[sel].contiguous(), opt)
    ted = torch.from_numpy(te).cuda()
    pred = mlp.forward(feat[ted].contiguous())
    rmse_mlp = float(torch.sqrt(((pred - y[ted]) ** 2).mean()))
    rmse_idw = float(torch.sqrt(((idw[ted] - y[ted]) ** 2).mean()))
    print(f"held-out RMSE (m/s): MLP {rmse_mlp:.3f}  IDW {rmse_idw:.3f}")
    assert rmse_mlp < rmse_idw
    assert rmse_mlp > 0.9  # the noise floor is 1 m/s per component


def test_training_steps_replayed_from_a_cuda_graph_match_eager_steps():
    # The AdamW step count lives on the device, so a captured sequence of
    # train steps replays with the right bias corrections.
    rng = np.random.default_rng(11)
    xs = [torch.from_numpy(rng.normal(0, 1, size=(640, 96)).astype(np.float32)).to(torch.bfloat16).cuda()
          for _ in range(4)]
    ts = [torch.from_numpy(rng.normal(0, 1, size=(640, 2)).astype(np.float32)).cuda() for _ in range(4)]
    opt = tnn.AdamW(lr=2e-3, weight_decay=1e-2)
    eager = tnn.MLP(96, 128, seed=21)
    for x, t in zip(xs, ts):
        eager.train_step(x, t, opt)
    graphed = tnn.MLP(96, 128, seed=21)
    graphed.gradients(xs[0], ts[0])  # sizes the workspace; no update
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for x, t in zip(xs, ts):
            graphed.train_step(x, t, opt)
    g.replay()
    torch.cuda.synchronize()
    a = eager.get_params(with_moments=True)
    b = graphed.get_params(with_moments=True)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3] == b[3] == 4
    g.replay()  # four more steps
    assert graphed.get_params(with_moments=True)[3] == 8


def _gka_setup(n_flights=60, k=16, lag=600.0):
    wl = synth.flights(n_flights, 80, seed=synth.SEED_LEARNED + 3, n_routes=6)
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 16)
    idx, _ = tnn.tnn_knn(ix, k, lag)
    return wl, ix, idx, torch.from_numpy(wl.wind).cuda()


def test_gka_forward_matches_oracle():
    wl, ix, idx, wind = _gka_setup()
    sig = np.array([0.05, 4.0, 1e-4], np.float32)
    g = tnn.GKA(sig)
    uv = g.forward(ix, wind, idx).cpu().numpy()
    ref, _ = nc.gka_forward(wl.xyzt, wl.wind, wl.xyzt, idx.cpu().numpy(), np.log(sig.astype(np.float64)))
    nan = np.isnan(ref).any(axis=1)
    assert nan.any() and not nan.all()  # some queries have no causal point
    assert np.isnan(uv[nan]).all()
    np.testing.assert_allclose(uv[~nan], ref[~nan], rtol=1e-4, atol=1e-4)
    # external queries
    q = wl.xyzt[::7].copy()
    q[:, 0] += 0.3
    qi, _ = tnn.tnn_knn(ix, 16, 600.0, q=torch.from_numpy(q).cuda())
    uq = g.forward(ix, wind, qi, q=torch.from_numpy(q).cuda()).cpu().numpy()
    rq, _ = nc.gka_forward(wl.xyzt, wl.wind, q, qi.cpu().numpy(), np.log(sig.astype(np.float64)))
    ok = ~np.isnan(rq).any(axis=1)
    np.testing.assert_allclose(uq[ok], rq[ok], rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("k", [5, 48])
def test_gka_forward_other_context_sizes(k):
    """Contexts narrower than a warp (two queries per warp) and wider than
    one (one query per warp, two neighbours per lane) against the oracle."""
    wl, ix, _, wind = _gka_setup()
    sig = np.array([0.05, 4.0, 1e-4], np.float32)
    g = tnn.GKA(sig)
    gm = tnn.GKAMLP(sig, hidden=16, seed=3)
    idx, _ = tnn.tnn_knn(ix, k, 600.0)
    uv = g.forward(ix, wind, idx).cpu().numpy()
    ref, _ = nc.gka_forward(wl.xyzt, wl.wind, wl.xyzt, idx.cpu().numpy(), np.log(sig.astype(np.float64)))
    ok = ~np.isnan(ref).any(axis=1)
    assert np.isnan(uv[~ok]).all()
    np.testing.assert_allclose(uv[ok], ref[ok], rtol=1e-4, atol=1e-4)
    w, _ = gm.get_params()
    lo, hi = wl.xyzt.min(axis=0), wl.xyzt.max(axis=0)
    um = gm.forward(ix, wind, idx).cpu().numpy()
    rm = nc.gkamlp_forward(wl.xyzt, wl.wind, wl.xyzt, idx.cpu().numpy(), w, 16, lo, hi)
    np.testing.assert_allclose(um[ok], rm[ok], rtol=1e-4, atol=1e-4)


def test_gka_gradient_and_adam_step_match_oracle():
    wl, ix, idx, wind = _gka_setup()
    idx_h = idx.cpu().numpy()
    full = (idx_h >= 0).all(axis=1)
    rows = np.nonzero(full)[0][:1500].astype(np.int32)
    rows_d = torch.from_numpy(rows).cuda()
    sig = np.array([0.05, 4.0, 1e-4], np.float32)
    g = tnn.GKA(sig)
    loss, grad = g.gradients(ix, wind, rows_d, idx)
    th = np.log(sig.astype(np.float64))
    rl, rg = nc.gka_loss_grad(wl.xyzt, wl.wind, rows, idx_h, th)
    assert float(loss.item()) == pytest.approx(rl, rel=1e-4)
    np.testing.assert_allclose(grad.cpu().numpy(), rg, rtol=2e-3, atol=1e-6 * np.abs(rg).max())
    opt = tnn.AdamW(lr=0.05, weight_decay=0.0)
    mm = np.zeros(3)
    vv = np.zeros(3)
    tk = th.copy()
    for t in range(1, 4):
        _, gt = nc.gka_loss_grad(wl.xyzt, wl.wind, rows, idx_h, tk)
        g.train_step(ix, wind, rows_d, idx, opt)
        tk, mm, vv = nc.adamw_step(tk, gt, mm, vv, t, lr=opt.lr, beta1=opt.beta1, beta2=opt.beta2,
                                   eps=opt.eps, wd=0.0)
        got, step = g.get_params()
        assert step == t
        np.testing.assert_allclose(np.log(got.astype(np.float64)), tk, rtol=0, atol=2e-4)


def test_gka_training_lowers_the_loss():
    wl, ix, idx, wind = _gka_setup(n_flights=120, k=32, lag=1800.0)
    full = (idx >= 0).all(dim=1).nonzero().flatten().to(torch.int32)
    g = tnn.GKA((1.0, 10.0, 0.01))
    l0, _ = g.gradients(ix, wind, full, idx)
    opt = tnn.AdamW(lr=0.05, weight_decay=0.0)
    for _ in range(150):
        g.train_step(ix, wind, full, idx, opt)
    l1, g1 = g.gradients(ix, wind, full, idx)
    # the context is at least 30 min old: the scales gain little, but they
    # must gain something and approach a stationary point
    assert float(l1.item()) < (1 - 1e-3) * float(l0.item())
    _, g0 = tnn.GKA((1.0, 10.0, 0.01)).gradients(ix, wind, full, idx)
    assert float(g1.norm()) < float(g0.norm())


def test_gkamlp_starts_as_gka_and_matches_oracle():
    wl, ix, idx, wind = _gka_setup()
    sig = np.array([0.05, 4.0, 1e-4], np.float32)
    g = tnn.GKAMLP(sig, hidden=16, seed=3)
    plain = tnn.GKA(sig)
    a = g.forward(ix, wind, idx).cpu().numpy()
    b = plain.forward(ix, wind, idx).cpu().numpy()
    ok = ~np.isnan(b).any(axis=1)
    np.testing.assert_allclose(a[ok], b[ok], rtol=2e-5, atol=2e-5)
    # a model with non-zero output weights against the oracle
    rng = np.random.default_rng(4)
    w, _ = g.get_params()
    H = 16
    w[4 * H:7 * H] = (0.5 * rng.normal(size=3 * H)).astype(np.float32)
    g.set_params(w)
    lo, hi = wl.xyzt.min(axis=0), wl.xyzt.max(axis=0)
    got = g.forward(ix, wind, idx).cpu().numpy()
    ref = nc.gkamlp_forward(wl.xyzt, wl.wind, wl.xyzt, idx.cpu().numpy(), w, H, lo, hi)
    ok = ~np.isnan(ref).any(axis=1)
    assert np.isnan(got[~ok]).all()
    np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-4, atol=2e-4)


def test_gkamlp_gradient_and_adam_steps_match_oracle():
    wl, ix, idx, wind = _gka_setup()
    idx_h = idx.cpu().numpy()
    rows = np.nonzero((idx_h >= 0).all(axis=1))[0][:1500].astype(np.int32)
    rows_d = torch.from_numpy(rows).cuda()
    H = 8
    g = tnn.GKAMLP((0.05, 4.0, 1e-4), hidden=H, seed=5)
    w, _ = g.get_params()
    w[4 * H:7 * H] = (0.3 * np.random.default_rng(6).normal(size=3 * H)).astype(np.float32)
    g.set_params(w)
    lo, hi = wl.xyzt.min(axis=0), wl.xyzt.max(axis=0)
    loss, grad = g.gradients(ix, wind, rows_d, idx)
    rl, rg = nc.gkamlp_loss_grad(wl.xyzt, wl.wind, rows, idx_h, w, H, lo, hi)
    assert float(loss.item()) == pytest.approx(rl, rel=1e-4)
    np.testing.assert_allclose(grad.cpu().numpy(), rg, rtol=5e-3, atol=2e-3 * np.abs(rg).max())
    opt = tnn.AdamW(lr=0.02, weight_decay=0.0)
    wk = w.astype(np.float64)
    mm = np.zeros_like(wk)
    vv = np.zeros_like(wk)
    for t in range(1, 3):
        _, gt = nc.gkamlp_loss_grad(wl.xyzt, wl.wind, rows, idx_h, wk, H, lo, hi)
        g.train_step(ix, wind, rows_d, idx, opt)
        wk, mm, vv = nc.adamw_step(wk, gt, mm, vv, t, lr=opt.lr, beta1=opt.beta1, beta2=opt.beta2,
                                   eps=opt.eps, wd=0.0)
        got, step = g.get_params()
        assert step == t
        # Adam normalises each coordinate: compare where the gradient is not tiny
        big = np.abs(gt) > 1e-3 * np.abs(gt).max()
        np.testing.assert_allclose(got[big], wk[big], rtol=0, atol=3e-3)


def test_window_average_matches_oracle():
    """The hour average of Sec. 4.1 ([t - 1 h 30, t - 30 min]) and the day
    average against the float64 oracle, self-queries and external ones
    (including windows that hold no point)."""
    wl = synth.flights(300, 200, seed=77, n_routes=6)  # 60,000 points over 6 h
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 20)
    wind = torch.from_numpy(wl.wind).cuda()
    hour = tnn.tnn_window_average(ix, wind).cpu().numpy()
    sel = synth.query_sample(wl.n, 3000, seed=4)
    ref = nc.window_average(wl.xyzt, wl.wind, wl.xyzt[sel])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(hour[sel]), nan)
    assert nan.any() and not nan.all()
    np.testing.assert_allclose(hour[sel][~nan], ref[~nan], rtol=1e-6, atol=1e-6)
    # external queries at other times, and the day average (every point)
    rng = np.random.default_rng(3)
    q = wl.xyzt[rng.choice(wl.n, 700, replace=False)].copy()
    q[:, 3] = rng.uniform(-1000.0, 30000.0, size=700).astype(np.float32)
    qd = torch.from_numpy(q).cuda()
    got = tnn.tnn_window_average(ix, wind, 7200.0, 600.0, q=qd).cpu().numpy()
    ref = nc.window_average(wl.xyzt, wl.wind, q, 7200.0, 600.0)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    np.testing.assert_allclose(got[~nan], ref[~nan], rtol=1e-6, atol=1e-6)
    day = tnn.tnn_window_average(ix, wind, float("inf"), float("-inf"), q=qd[:5]).cpu().numpy()
    np.testing.assert_allclose(day, np.repeat(wl.wind.astype(np.float64).mean(axis=0)[None], 5, axis=0),
                               rtol=1e-6)


def test_checkpoint_rejects_other_shapes_and_truncated_files(tmp_path):
    m = tnn.MLP(64, 64, seed=1)
    p = tmp_path / "a.bin"
    m.save(str(p))
    other = tnn.MLP(64, 128, seed=1)
    with pytest.raises(tnn.TNNError) as ei:
        other.load(str(p))
    assert ei.value.status == 1
    raw = p.read_bytes()
    (tmp_path / "cut.bin").write_bytes(raw[:-4])
    with pytest.raises(tnn.TNNError):
        m.load(str(tmp_path / "cut.bin"))
    # the file layout: five little-endian int64, then three float32 blocks
    hdr = np.frombuffer(raw[:40], dtype="<i8")
    assert hdr.tolist() == [0x544E4E4D, 1, 64, 64, 0]
    assert len(raw) == 40 + 3 * 4 * m.n_params
    np.testing.assert_array_equal(np.frombuffer(raw[40:40 + 4 * m.n_params], dtype="<f4"), m.get_params())
