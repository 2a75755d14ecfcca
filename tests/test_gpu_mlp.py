"""Parity of the learned proposal's CUDA path (pump_mlp_*) with the float64 oracle (oracle/mlp.py).

Tolerances.  The device sums products in FP32 where the oracle sums exactly (relative difference
about 1e-7, the median error seen).  The BF16 rounding of a hidden activation or of a backward
gradient can then land on the other side of a rounding boundary (about once per 3e4 roundings),
moving that value by one BF16 unit, at most 2^-8 |h|.  With activations up to |h| ~ 8 and He-scaled
weights up to sqrt(6/256) ~ 0.15, one flip in the last hidden layer moves an output by up to
2^-8 * 8 * 0.15 ~ 5e-3; the bound 1e-2 admits two such flips in one row.  The median error is bound
at 2e-5, which a wrong index, operand or epilogue would exceed by orders of magnitude."""
import numpy as np
import pytest

from oracle import mlp as orc
from paper_1607_06886_gb300 import pump

pytestmark = pytest.mark.gpu

DIMS = [224, 256, 256, 256, 16]
VMAX = 0.1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    yield


def he_params(dims, seed, bias_scale=0.05):
    g = np.random.default_rng(seed)
    layers = [(g.uniform(-1, 1, (dims[l + 1], dims[l])) * np.sqrt(6.0 / dims[l]),
               bias_scale * g.standard_normal(dims[l + 1])) for l in range(len(dims) - 1)]
    return orc.join_params(layers).astype(np.float32)


def env_feats(n_env, seed):
    g = np.random.default_rng(seed)
    f = np.zeros((n_env, orc.FEAT_ENV), np.float32)
    for e in range(n_env):
        nb = g.integers(3, 33)
        lo = g.uniform(0, 0.8, (nb, 3))
        f[e, :nb * 6] = np.concatenate([lo, lo + g.uniform(0.02, 0.2, (nb, 3))], axis=1).ravel()
        f[e, 192:198] = [0.1, 0.1, 0.1, 0, 0, 0]
        f[e, 198:204] = [0.9, 0.9, 0.9, 0, 0, 0]
    return f


def targets(n, T, seed):
    g = np.random.default_rng(seed)
    t = np.concatenate([g.uniform(0, 1, (n, T, 3)), g.uniform(-VMAX, VMAX, (n, T, 3))], axis=2).astype(np.float32)
    nt = g.integers(1, T + 1, size=n).astype(np.int32)
    return t, nt


def model_with(params, dims=DIMS):
    m = pump.MLP(dims, 0)
    m.set_params(params)
    return m


def close(a, b, atol, med):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    assert d.max() <= atol, (d.max(), atol)
    assert np.median(d) <= med, (np.median(d), med)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("B", [1, 37, 48, 272, 1040])
def test_forward_matches_oracle(B):
    p = he_params(DIMS, 1)
    x = np.random.default_rng(2).uniform(-1, 1, (B, DIMS[0])).astype(np.float32)
    m = model_with(p)
    y = m.forward(x)
    o, _ = orc.forward(p.astype(np.float64), DIMS, x)
    close(y, o, atol=1e-2, med=2e-5)
    m.close()


def test_forward_other_shapes():
    dims = [32, 48, 16]           # widths that are not multiples of the 64-wide tile
    p = he_params(dims, 3)
    x = np.random.default_rng(4).standard_normal((80, 32)).astype(np.float32)
    m = model_with(p, dims)
    o, _ = orc.forward(p.astype(np.float64), dims, x)
    close(m.forward(x), o, atol=1e-2, med=2e-5)
    m.close()


@pytest.mark.parametrize("B", [16, 200, 2048])
def test_gradients_match_oracle(B):
    p = he_params(DIMS, 5)
    g = np.random.default_rng(6)
    x = g.uniform(-1, 1, (B, DIMS[0])).astype(np.float32)
    dy = (g.standard_normal((B, DIMS[-1])) / B).astype(np.float32)
    m = model_with(p)
    gg = m.gradients(x, dy)
    o, hs = orc.forward(p.astype(np.float64), DIMS, x)
    go = orc.backward(p.astype(np.float64), DIMS, hs, dy)
    for l, ((Wg, bg), (Wo, bo)) in enumerate(zip(orc.split_params(gg, DIMS), orc.split_params(go, DIMS))):
        for a, b in ((Wg, Wo), (bg, bo)):
            scale = np.abs(b).max()
            assert np.abs(a - b).max() <= 2e-2 * scale, (l, np.abs(a - b).max(), scale)
            assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b), (l, np.linalg.norm(a - b), np.linalg.norm(b))
    # parameters untouched, and the library's vector length is the oracle's count
    assert m.n_params == orc.param_count(DIMS) == len(p)
    assert np.array_equal(m.get_params()[0], p)
    m.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_train_step_matches_oracle(kind):
    B, T = 96, 6
    p = he_params(DIMS, 7)
    g = np.random.default_rng(8)
    x = g.uniform(-1, 1, (B, DIMS[0])).astype(np.float32)
    x[:, orc.FEAT_ENV] = g.standard_normal(B)   # the first latent (read by the path-indexed loss)
    tg, nt = targets(B, T, 9)
    nt[5] = 0                       # a row without targets adds nothing
    nt[6] = 1                       # a one-state path
    m = model_with(p)
    m.set_loss(kind, orc.FEAT_ENV)
    lr = 1e-3
    loss = m.train_step(x, tg, nt, lr, VMAX)
    w1, steps = m.get_params()
    assert steps == 1
    o, hs = orc.forward(p.astype(np.float64), DIMS, x)
    lo, go = orc.wta_loss(o, tg, nt, VMAX, kind, hs[0][:, orc.FEAT_ENV])
    assert loss == pytest.approx(lo.mean(), rel=2e-3)
    grad = orc.backward(p.astype(np.float64), DIMS, hs, go)
    w_orc, _, _ = orc.adam(p.astype(np.float64), grad, 0 * grad, 0 * grad, 1, lr)
    d = np.abs(w1 - w_orc)
    # first Adam step moves each weight by lr * g / (|g| + eps): by lr wherever |g| is clearly nonzero
    clear = np.abs(grad) > 1e-2 * np.abs(grad).max()
    assert clear.sum() > 1000
    assert d[clear].max() <= 1e-2 * lr, d[clear].max()
    assert d.max() <= 2.0 * lr + 1e-6
    m.close()


def test_assemble_matches_oracle_draws():
    n_env, B = 23, 300
    f = env_feats(n_env, 10)
    tg, nt = targets(n_env, 8, 11)
    m = pump.MLP(DIMS, 0)
    m.set_data(f, tg, nt)
    for t in (0, 7, 123456):
        x, env = m.assemble(B, t, 99)
        z, env_o = orc.train_draws(99, t, B, n_env)
        assert np.array_equal(env, env_o)
        xo = orc.bf16(orc.assemble(f, env_o, z, DIMS[0]))
        # features and padding bit for bit; normals within one BF16 unit (device Box-Muller is FP32)
        assert np.array_equal(x[:, :orc.FEAT_ENV], xo[:, :orc.FEAT_ENV])
        assert not x[:, orc.FEAT_ENV + 8:].any()
        zd = np.abs(x[:, orc.FEAT_ENV:orc.FEAT_ENV + 8] - xo[:, orc.FEAT_ENV:orc.FEAT_ENV + 8])
        assert np.all(zd <= 2.0 ** -7 * np.maximum(np.abs(xo[:, orc.FEAT_ENV:orc.FEAT_ENV + 8]), 1e-30))
        assert (zd == 0).mean() > 0.99
    m.close()


def test_propose_matches_oracle():
    p = he_params(DIMS, 12, bias_scale=0.5)
    f = env_feats(1, 13)[0]
    m = model_with(p)
    for count in (1, 100, 2000):
        s = m.propose(f, count, 5, VMAX)
        so = orc.propose(p.astype(np.float64), DIMS, f, count, 5, VMAX)
        close(s, so, atol=2e-3, med=1e-5)
        assert np.all((s[:, :3] >= 0) & (s[:, :3] <= 1)) and np.all(np.abs(s[:, 3:]) <= VMAX)
    m.close()


# ---------------------------------------------------------------------------
def small_problem(seed=20, n_env=40, T=5):
    f = env_feats(n_env, seed)
    tg, nt = targets(n_env, T, seed + 1)
    return f, tg, nt


def test_training_loop_lowers_loss_and_is_deterministic():
    f, tg, nt = small_problem()
    a = pump.MLP(DIMS, 3)
    b = pump.MLP(DIMS, 3)
    for m in (a, b):
        m.set_data(f, tg, nt)
    tr = a.train(256, 300, 1e-3, VMAX, 7)
    assert np.all(np.isfinite(tr))
    assert tr[-30:].mean() < 0.5 * tr[:10].mean(), (tr[:10].mean(), tr[-30:].mean())
    # the same steps split over two calls: bit for bit (counter-based draws, fixed summation order)
    t1 = b.train(256, 120, 1e-3, VMAX, 7)
    t2 = b.train(256, 180, 1e-3, VMAX, 7)
    assert np.array_equal(np.concatenate([t1, t2]), tr)
    pa, sa = a.get_params()
    pb, sb = b.get_params()
    assert sa == sb == 300 and np.array_equal(pa, pb)
    a.close()
    b.close()


def test_training_loop_step_equals_explicit_step():
    f, tg, nt = small_problem(30)
    a = pump.MLP(DIMS, 4)
    b = pump.MLP(DIMS, 4)
    a.set_data(f, tg, nt)
    b.set_data(f, tg, nt)
    B = 512
    x, env = b.assemble(B, 0, 11)
    la = a.train(B, 1, 2e-3, VMAX, 11)[0]
    lb = b.train_step(x, tg[env], nt[env], 2e-3, VMAX)
    assert la == lb
    assert np.array_equal(a.get_params()[0], b.get_params()[0])
    a.close()
    b.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_training_loop_matches_oracle_steps(kind):
    dims = [64, 64, 64, 16]
    F = dims[0] - 8
    g = np.random.default_rng(40)
    n_env, T = 12, 4
    f = g.uniform(0, 1, (n_env, F)).astype(np.float32)
    tg, nt = targets(n_env, T, 41)
    p = he_params(dims, 42)
    m = model_with(p, dims)
    m.set_loss(kind, F)
    m.set_data(f, tg, nt)
    tr = m.train(64, 5, 1e-3, VMAX, 3)
    st = {"w": p.astype(np.float64), "m": np.zeros(p.size), "v": np.zeros(p.size), "t": 0}
    lo = [orc.train_step(st, dims, f, tg, nt, 64, 3, 1e-3, VMAX, kind) for _ in range(5)]
    assert np.allclose(tr, lo, rtol=5e-3, atol=1e-6), (tr, lo)
    w, steps = m.get_params()
    assert steps == 5
    # after a few steps each weight has moved by up to ~5 lr; the paths agree to a fraction of lr
    assert np.median(np.abs(w - st["w"])) < 1e-2 * 1e-3
    m.close()


def test_invalid_arguments():
    with pytest.raises(pump.PumpError):
        pump.MLP([224, 250, 16])
    m = pump.MLP([32, 32, 16])
    with pytest.raises(pump.PumpError):
        m.set_params(np.zeros(3, np.float32))
    with pytest.raises(pump.PumpError):
        m.train(16, 1, 1e-3, VMAX, 0)            # no training set
    with pytest.raises(pump.PumpError):
        m.propose(np.zeros(30, np.float32), 4, 0, VMAX)  # 30 + 8 > 32
    with pytest.raises(pump.PumpError):
        m.set_loss(2, 0)
    with pytest.raises(pump.PumpError):
        m.set_loss(1, 32)
    m.close()
