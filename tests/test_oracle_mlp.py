"""Pins of the learned-proposal oracle (oracle/mlp.py) against what mathematics and libraries fix:
bfloat16 rounding against torch's conversion, closed-form forward passes, analytic gradients
against central finite differences, Adam's constant-gradient closed form, the winner-take-all rule
on hand-built cases, the draws' distributions, and a training run that lowers the loss."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------------------
def test_bf16_matches_torch_on_random_values():
    x = _rng(0).standard_normal(200000).astype(np.float32) * np.float32(3.0)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_bf16_ties_round_to_even():
    # patterns whose dropped half is exactly 0x8000: ties; kept low bit even -> down, odd -> up
    hi = _rng(1).integers(0x3F00, 0x4100, size=4096).astype(np.uint32)
    x = ((hi << 16) | 0x8000).astype(np.uint32).view(np.float32)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = mlp.bf16(x)
    assert np.array_equal(got, ref)
    even = (hi & 1) == 0
    assert np.all(got[even] < x[even]) and np.all(got[~even] > x[~even])


def test_bf16_keeps_representable_values():
    x = np.arange(-256, 257, dtype=np.float64) / 64.0
    assert np.array_equal(mlp.bf16(x), x)


# ---------------------------------------------------------------------------
def _identity_net(d=16, shift=0.25, gain=2.0, out_bias=0.1):
    W0 = np.eye(d)
    b0 = np.full(d, -shift)
    W1 = gain * np.eye(d)
    b1 = np.full(d, out_bias)
    return mlp.join_params([(W0, b0), (W1, b1)]), [d, d, d]


def test_forward_closed_form_relu():
    flat, dims = _identity_net()
    x = _rng(2).integers(0, 64, size=(32, 16)) / 64.0   # exact in bfloat16
    o, hs = mlp.forward(flat, dims, x)
    assert np.array_equal(o, 2.0 * np.maximum(x - 0.25, 0.0) + 0.1)
    assert np.array_equal(hs[1], np.maximum(x - 0.25, 0.0))


def test_forward_rounds_inputs_and_weights_to_bf16():
    d = 16
    W = np.zeros((d, d))
    W[0, 0] = 1.0 + 2.0 ** -10        # not representable: rounds to 1.0
    flat = mlp.join_params([(W, np.zeros(d))])
    x = np.zeros((16, d))
    x[:, 0] = 1.0 + 3 * 2.0 ** -9     # 0.75 ulp above 1: rounds up to 1 + 2^-7
    o, _ = mlp.forward(flat, [d, d], x)
    assert np.allclose(o[:, 0], 1.0 + 2.0 ** -7, rtol=0, atol=0)
    o64, _ = mlp.forward(flat, [d, d], x, quant=False)
    assert o64[0, 0] == (1.0 + 2.0 ** -10) * (1.0 + 3 * 2.0 ** -9)


def test_squash_limits():
    o = np.zeros((2, 16))
    o[1, :6] = 50.0
    s = mlp.squash(o, 0.1)
    assert np.allclose(s[0], [0.5, 0.5, 0.5, 0, 0, 0])
    assert np.allclose(s[1], [1, 1, 1, 0.1, 0.1, 0.1])


# ---------------------------------------------------------------------------
def _random_net(dims, seed):
    g = _rng(seed)
    layers = [(g.standard_normal((dims[l + 1], dims[l])) / np.sqrt(dims[l]), 0.1 * g.standard_normal(dims[l + 1]))
              for l in range(len(dims) - 1)]
    return mlp.join_params(layers)


def _fd(fun, theta, h=1e-6):
    g = np.zeros_like(theta)
    for k in range(len(theta)):
        e = np.zeros_like(theta)
        e[k] = h
        g[k] = (fun(theta + e) - fun(theta - e)) / (2 * h)
    return g


@pytest.mark.parametrize("dims", [[16, 32, 16], [16, 16, 32, 16]])
def test_backward_matches_finite_differences(dims):
    theta = _random_net(dims, 3)
    x = _rng(4).standard_normal((16, dims[0]))
    gout = _rng(5).standard_normal((16, dims[-1]))
    o, hs = mlp.forward(theta, dims, x, quant=False)
    # keep away from ReLU kinks so the finite difference sees one linear piece
    pre = []
    h = x
    for W, b in mlp.split_params(theta, dims)[:-1]:
        p = h @ W.T + b
        pre.append(p)
        h = np.maximum(p, 0)
    assert min(np.abs(p).min() for p in pre) > 1e-4
    ana = mlp.backward(theta, dims, hs, gout, quant=False)
    num = _fd(lambda t: float((mlp.forward(t, dims, x, quant=False)[0] * gout).sum()), theta)
    assert np.allclose(ana, num, rtol=1e-6, atol=1e-7)


def test_wta_picks_nearest_target_and_gradient_matches_fd():
    vmax = 0.1
    g = _rng(6)
    B, T = 16, 5
    o = g.standard_normal((B, 16)) * 0.5
    tg = np.concatenate([g.uniform(0, 1, (B, T, 3)), g.uniform(-vmax, vmax, (B, T, 3))], axis=2)
    n_t = g.integers(1, T + 1, size=B)
    n_t[3] = 0
    loss, grad = mlp.wta_loss(o, tg, n_t, vmax)
    s = mlp.squash(o, vmax)
    for r in range(B):
        if n_t[r] == 0:
            assert loss[r] == 0 and not grad[r].any()
            continue
        d = [((s[r] - tg[r, p]) ** 2).sum() for p in range(n_t[r])]
        assert loss[r] == pytest.approx(min(d), rel=1e-12)
    assert not grad[:, 6:].any()
    num = _fd(lambda v: float(mlp.wta_loss(v.reshape(B, 16), tg, n_t, vmax)[0].mean()), o.ravel())
    assert np.allclose(grad.ravel(), num, rtol=1e-5, atol=1e-9)


def test_wta_hand_example():
    # output squashes to (0.5, 0.5, 0.5, 0, 0, 0); the second target is nearer
    o = np.zeros((1, 16))
    tg = np.array([[[0.9, 0.5, 0.5, 0, 0, 0], [0.5, 0.5, 0.7, 0, 0, 0.05]]])
    loss, g = mlp.wta_loss(o, tg, [2], 0.1)
    assert loss[0] == pytest.approx(0.2 ** 2 + 0.05 ** 2, rel=1e-12)
    # d/do of (0.5 + 0.5 tanh o - 0.7)^2 at o = 0: 2 (-0.2) 0.5; velocity: 2 (-0.05) 0.1
    assert g[0, 2] == pytest.approx(-0.2, rel=1e-12)
    assert g[0, 5] == pytest.approx(-0.01, rel=1e-12)
    assert g[0, 0] == 0 and g[0, 3] == 0


def test_loss_gradient_through_network_matches_fd():
    dims = [16, 32, 16]
    theta = _random_net(dims, 7)
    g = _rng(8)
    B, T, vmax = 16, 4, 0.1
    x = g.standard_normal((B, 16))
    tg = np.concatenate([g.uniform(0, 1, (B, T, 3)), g.uniform(-vmax, vmax, (B, T, 3))], axis=2)
    n_t = np.full(B, T)

    def L(t):
        o, _ = mlp.forward(t, dims, x, quant=False)
        return float(mlp.wta_loss(o, tg, n_t, vmax)[0].mean())

    o, hs = mlp.forward(theta, dims, x, quant=False)
    _, go = mlp.wta_loss(o, tg, n_t, vmax)
    ana = mlp.backward(theta, dims, hs, go, quant=False)
    assert np.allclose(ana, _fd(L, theta), rtol=1e-5, atol=1e-9)


# ---------------------------------------------------------------------------
def test_adam_constant_gradient_steps_by_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    w = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 6):
        w_new, m, v = mlp.adam(w, g, m, v, t, lr=0.01)
        # with a constant gradient the bias-corrected moments are g and g^2 exactly
        assert np.allclose(w_new - w, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        w = w_new


def test_adam_zero_gradient_keeps_weights():
    w = np.array([1.0, -2.0])
    w2, m, v = mlp.adam(w, np.zeros(2), np.zeros(2), np.zeros(2), 1, 0.1)
    assert np.array_equal(w2, w)


# ---------------------------------------------------------------------------
def test_draws_are_standard_normal_and_envs_uniform():
    from scipy import stats
    z, env = mlp.train_draws(11, 5, 40000, 7)
    for j in range(8):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-3
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(8)).max() < 0.03
    cnt = np.bincount(env, minlength=7)
    assert stats.chisquare(cnt).pvalue > 1e-3
    assert env.min() >= 0 and env.max() < 7


def test_draws_depend_on_step_and_stream_only_through_the_counter():
    a, ea = mlp.train_draws(3, 0, 64, 5)
    b, eb = mlp.train_draws(3, 0, 64, 5)
    c, _ = mlp.train_draws(3, 1, 64, 5)
    assert np.array_equal(a, b) and np.array_equal(ea, eb)
    assert not np.array_equal(a, c)
    # rows are independent of the batch size (counter-based)
    d, ed = mlp.train_draws(3, 0, 16, 5)
    assert np.array_equal(d, a[:16]) and np.array_equal(ed, ea[:16])
    p = mlp.proposal_latents(3, 64)
    assert not np.array_equal(p, a)


def test_env_features_layout():
    bx = np.arange(12, dtype=np.float64).reshape(2, 6)
    f = mlp.env_features(bx, np.arange(6) + 100, np.arange(6) + 200)
    assert f.shape == (204,)
    assert np.array_equal(f[:12], np.arange(12)) and not f[12:192].any()
    assert np.array_equal(f[192:198], np.arange(6) + 100) and np.array_equal(f[198:], np.arange(6) + 200)


def test_training_lowers_the_loss():
    dims = [32, 32, 32, 16]
    g = _rng(9)
    n_env, T = 8, 4
    feat = np.zeros((n_env, 24))
    feat[:, :6] = g.uniform(0, 1, (n_env, 6))
    tg = np.concatenate([g.uniform(0, 1, (n_env, T, 3)), g.uniform(-0.1, 0.1, (n_env, T, 3))], axis=2)
    st = {"w": _random_net(dims, 10), "m": None, "v": None, "t": 0}
    st["m"] = np.zeros_like(st["w"])
    st["v"] = np.zeros_like(st["w"])
    losses = [mlp.train_step(st, dims, feat, tg, np.full(n_env, T), 32, 1, 3e-3, 0.1) for _ in range(150)]
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:10])


# ---------------------------------------------------------------------------
def test_path_point_walks_the_polyline():
    tg = np.array([[0.0] * 6, [1.0] * 6, [1.0, 3.0, 1.0, 1.0, 1.0, 1.0]])
    assert np.array_equal(mlp.path_point(tg, 3, 0.0), tg[0])
    assert np.allclose(mlp.path_point(tg, 3, 0.25), 0.5 * tg[1])
    assert np.allclose(mlp.path_point(tg, 3, 0.5), tg[1])
    assert np.allclose(mlp.path_point(tg, 3, 0.75), [1, 2, 1, 1, 1, 1])
    assert np.allclose(mlp.path_point(tg, 3, 1.0), tg[2])
    assert np.array_equal(mlp.path_point(tg, 1, 0.7), tg[0])


def test_normal_cdf_matches_scipy():
    from scipy import stats
    z = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.normal_cdf(z), stats.norm.cdf(z), rtol=1e-12, atol=1e-15)


def test_path_indexed_loss_and_gradient():
    vmax = 0.1
    g = _rng(12)
    B, T = 16, 5
    o = g.standard_normal((B, 16)) * 0.5
    tg = np.concatenate([g.uniform(0, 1, (B, T, 3)), g.uniform(-vmax, vmax, (B, T, 3))], axis=2)
    n_t = g.integers(1, T + 1, size=B)
    n_t[2] = 0
    z0 = g.standard_normal(B)
    loss, grad = mlp.wta_loss(o, tg, n_t, vmax, kind=1, z0=z0)
    s = mlp.squash(o, vmax)
    from scipy import stats
    for r in range(B):
        if n_t[r] == 0:
            assert loss[r] == 0
            continue
        u = stats.norm.cdf(z0[r])
        y = mlp.path_point(tg[r], n_t[r], u)
        assert loss[r] == pytest.approx(((s[r] - y) ** 2).sum(), rel=1e-12)
    num = _fd(lambda v: float(mlp.wta_loss(v.reshape(B, 16), tg, n_t, vmax, 1, z0)[0].mean()), o.ravel())
    assert np.allclose(grad.ravel(), num, rtol=1e-5, atol=1e-9)


def test_path_indexed_training_spreads_outputs_along_the_path():
    # one environment whose targets are two far-apart states: winner-take-all may settle on one,
    # the path-indexed loss has to produce both ends as the first latent varies
    dims = [32, 64, 64, 16]
    feat = np.zeros((1, 24))
    tg = np.array([[[0.2, 0.2, 0.2, 0, 0, 0], [0.8, 0.8, 0.8, 0, 0, 0]]])
    st = {"w": _random_net(dims, 13), "t": 0}
    st["m"] = np.zeros_like(st["w"])
    st["v"] = np.zeros_like(st["w"])
    for _ in range(400):
        mlp.train_step(st, dims, feat, tg, [2], 64, 5, 3e-3, 0.1, kind=1)
    z = np.array([-2.5, 0.0, 2.5])
    x = np.zeros((3, 32))
    x[:, 24] = z
    o, _ = mlp.forward(st["w"], dims, x)
    pos = mlp.squash(o, 0.1)[:, 0]
    assert pos[0] < 0.3 and abs(pos[1] - 0.5) < 0.1 and pos[2] > 0.7, pos
