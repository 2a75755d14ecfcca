"""CPU oracle of the learned sampling proposal (an extension; the paper has no learning).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU baseline use this
module.  It restates, in numpy float64, what the proposal network and its training compute, with
the BF16 rounding written out at the points where the method stores BF16.  It shares no code with
the CUDA library; the random draws come from the oracle's own Philox4x64-10 (pump_oracle.c, O7).

Definitions (the method's, stated here once):

  Features   x = [boxes (32 x 6: lo, hi; zero rows past the scene's boxes), start (6), goal (6),
             z (8 standard normals), zeros] padded to dims[0].  The first 204 entries are the
             environment's; z is drawn per row.
  Network    h_0 = bf16(x); pre_l = W_l h_l + b_l; h_{l+1} = bf16(relu(pre_l)) for l < L-1;
             o = pre_{L-1}.  W_l (out x in) and b_l are FP32 master values; the products use
             bf16(W_l); sums are FP32 on the device, exact here.
  Squash     s_j = 0.5 + 0.5 tanh(o_j) for j < 3 (position in the unit cube),
             s_j = vmax tanh(o_j) for 3 <= j < 6 (velocity); outputs past 6 are unused.
  Loss       kind 0, winner takes all over a row's targets y_0 .. y_{n-1} (the states along a
             solution path, in path order): loss_r = min_p |s - y_p|^2 (first minimiser on
             ties).  Kind 1, path-indexed: u = Phi(z_0) (standard normal CDF of the row's first
             latent as the network sees it, i.e. after BF16 rounding), a = u (n - 1),
             i = min(floor(a), n - 2), f = a - i, target y(u) = y_i + f (y_{i+1} - y_i)
             (y_0 when n = 1); loss_r = |s - y(u)|^2.  The batch loss is the mean.
  Backward   g = bf16(d mean loss / d o); dW_l = g_l^T h_l, db_l = sum over rows of g_l,
             g_{l-1} = bf16((g_l bf16(W_l)) * [h_l > 0]).
  Adam       Kingma and Ba (2015) with bias correction: beta1 0.9, beta2 0.999, eps 1e-8.
  Draws      row r of draw set (t, stream): latents from Philox counter (t, r, stream, 0), key
             (seed, 1); the training row's environment from counter (t, r, stream + 1, 0).
             Training step t uses stream 0; the proposal for a query with seed s uses t = 0,
             stream 2, rows 0 .. count-1.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import cpu

N_BOX_SLOTS = 32
FEAT_ENV = N_BOX_SLOTS * 6 + 12   # 204 environment features
LATENT = 8
OUT_USED = 6
TRAIN_STREAM = 0
PROPOSAL_STREAM = 2


# ---------------------------------------------------------------------------
def bf16(x) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) from the float32 value, as float64.

    bfloat16 keeps the top 16 bits of the IEEE float32 pattern; rounding adds 0x7FFF plus the
    lowest kept bit before truncating.  NaN is not handled (the method never makes one)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split_params(flat: np.ndarray, dims: Sequence[int]) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Flat parameter vector (per layer W (out x in, row-major) then b) -> [(W, b)]."""
    out, off = [], 0
    for l in range(len(dims) - 1):
        i, o = dims[l], dims[l + 1]
        W = np.asarray(flat[off:off + i * o], np.float64).reshape(o, i)
        off += i * o
        b = np.asarray(flat[off:off + o], np.float64)
        off += o
        out.append((W, b))
    assert off == len(flat)
    return out


def join_params(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def param_count(dims: Sequence[int]) -> int:
    return sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))


# ---------------------------------------------------------------------------
def forward(flat, dims, x, quant: bool = True) -> Tuple[np.ndarray, List[np.ndarray]]:
    """Network outputs o (B x dims[-1]) and the layer inputs h_0 .. h_{L-1}.

    quant=False drops every BF16 rounding (a plain float64 network, for finite differences)."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    layers = split_params(flat, dims)
    h = q(x)
    hs = [h]
    for l, (W, b) in enumerate(layers):
        pre = h @ q(W).T + b
        if l + 1 < len(layers):
            h = q(np.maximum(pre, 0.0))
            hs.append(h)
        else:
            return pre, hs
    raise AssertionError


def squash(o, vmax: float) -> np.ndarray:
    o = np.asarray(o, np.float64)[:, :OUT_USED]
    s = np.empty_like(o)
    s[:, :3] = 0.5 + 0.5 * np.tanh(o[:, :3])
    s[:, 3:] = vmax * np.tanh(o[:, 3:])
    return s


def path_point(tg, n: int, u: float) -> np.ndarray:
    """The state at fraction u of the polyline y_0 .. y_{n-1} by node index (kind-1 target)."""
    tg = np.asarray(tg, np.float64)
    if n == 1:
        return tg[0].copy()
    a = u * (n - 1)
    i = min(int(math.floor(a)), n - 2)
    f = a - i
    return tg[i] + f * (tg[i + 1] - tg[i])


def normal_cdf(z) -> np.ndarray:
    return 0.5 * np.vectorize(math.erfc)(-np.asarray(z, np.float64) / math.sqrt(2.0))


def wta_loss(o, targets, n_targets, vmax: float, kind: int = 0, z0=None) -> Tuple[np.ndarray, np.ndarray]:
    """Per-row loss and d(mean loss)/d o (B x o.shape[1], zero past column 6).

    targets: (B, T, 6); row r uses its first n_targets[r] targets; a row without targets has
    loss 0 and no gradient.  kind 0: min_p |s - y_p|^2; kind 1: |s - y(Phi(z0[r]))|^2."""
    o = np.asarray(o, np.float64)
    B = o.shape[0]
    s = squash(o, vmax)
    loss = np.zeros(B)
    g = np.zeros_like(o)
    u = normal_cdf(z0) if kind == 1 else None
    for r in range(B):
        k = int(n_targets[r])
        if k <= 0:
            continue
        if kind == 0:
            d = ((s[r][None, :] - np.asarray(targets[r][:k], np.float64)) ** 2).sum(axis=1)
            p = int(np.argmin(d))  # first minimiser
            y = np.asarray(targets[r][p], np.float64)
            loss[r] = d[p]
        else:
            y = path_point(targets[r], k, float(u[r]))
            loss[r] = ((s[r] - y) ** 2).sum()
        th = np.tanh(o[r, :OUT_USED])
        ds = np.where(np.arange(OUT_USED) < 3, 0.5, vmax) * (1.0 - th * th)
        g[r, :OUT_USED] = 2.0 * (s[r] - y) * ds / B
    return loss, g


def backward(flat, dims, hs, g_out, quant: bool = True) -> np.ndarray:
    """Gradients (flat, parameter layout) of sum(g_out * o) given the forward's layer inputs."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    layers = split_params(flat, dims)
    grads = [None] * len(layers)
    g = q(g_out)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (g.T @ hs[l], g.sum(axis=0))
        if l > 0:
            g = q((g @ q(W)) * (hs[l] > 0))
    return join_params(grads)


def adam(w, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step t >= 1); returns new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
def env_features(boxes, start, goal) -> np.ndarray:
    """The 204 environment features: box rows (lo, hi) in the scene's order, zero rows up to 32,
    then the start and goal states."""
    bx = np.asarray(boxes, np.float64).reshape(-1, 6)
    if bx.shape[0] > N_BOX_SLOTS:
        raise ValueError("at most 32 boxes")
    f = np.zeros(FEAT_ENV)
    f[:bx.shape[0] * 6] = bx.ravel()
    f[N_BOX_SLOTS * 6:N_BOX_SLOTS * 6 + 6] = start
    f[N_BOX_SLOTS * 6 + 6:] = goal
    return f


def assemble(env_feat, env_idx, z, d0: int) -> np.ndarray:
    """Network inputs: row r = [env_feat[env_idx[r]], z[r], zeros] (width d0)."""
    F = np.asarray(env_feat, np.float64)
    x = np.zeros((len(env_idx), d0))
    x[:, :F.shape[1]] = F[np.asarray(env_idx)]
    x[:, F.shape[1]:F.shape[1] + LATENT] = z
    return x


def train_draws(seed: int, t: int, rows: int, n_env: int):
    """Latents and environments of training step t (stream 0)."""
    return cpu.mlp_draws(seed, t, TRAIN_STREAM, rows, n_env)


def proposal_latents(seed: int, count: int) -> np.ndarray:
    z, _ = cpu.mlp_draws(seed, 0, PROPOSAL_STREAM, count, 0)
    return z


def propose(flat, dims, env_feat_row, count: int, seed: int, vmax: float) -> np.ndarray:
    """Proposal states (count x 6) for one environment."""
    z = proposal_latents(seed, count)
    x = assemble(np.asarray(env_feat_row)[None, :], np.zeros(count, np.int64), z, dims[0])
    o, _ = forward(flat, dims, x)
    return squash(o, vmax)


def train_step(state: Dict, dims, env_feat, targets, n_targets, batch: int, seed: int, lr: float,
               vmax: float, kind: int = 0) -> float:
    """One training step in place on state = {w, m, v, t}: draws of step t (the count of steps
    taken before), forward, loss, backward, Adam.  Returns the mean loss."""
    t = int(state["t"])
    z, env = train_draws(seed, t, batch, len(env_feat))
    x = assemble(env_feat, env, z, dims[0])
    o, hs = forward(state["w"], dims, x)
    F = np.asarray(env_feat).shape[1]
    loss, g = wta_loss(o, np.asarray(targets)[env], np.asarray(n_targets)[env], vmax, kind, hs[0][:, F])
    grad = backward(state["w"], dims, hs, g)
    state["w"], state["m"], state["v"] = adam(state["w"], grad, state["m"], state["v"], t + 1, lr)
    state["t"] = t + 1
    return float(loss.mean())
