"""Pins of the CPU oracle against things other than itself (no GPU).

Each test ties one oracle function to a library routine, a closed form, an
invariant, a brute-force enumeration or a second independent restatement, so
that a dropped term, a wrong sign or a swapped index in the oracle fails here.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.interpolate
import scipy.linalg
import scipy.optimize
import scipy.stats

from oracle import cpu, naive
from paper_1607_06886_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ3 = math.sqrt(3.0)
A_CL = np.array([[0.0, 1.0], [-1.0, -SQ3]])


# --------------------------------------------------------------------------- O1
@pytest.mark.parametrize("dp", [[0.3, 0.0, 0.0], [0.1, -0.2, 0.05], [1.0, 1.0, 1.0], [1e-3, 0, 0]])
def test_steer_rest_to_rest_closed_form(dp):
    # at rest at both ends the optimum is tau = (36 |dp|^2)^(1/4), J = (4/3) tau
    x1 = np.r_[dp, 0, 0, 0]
    tau, J = cpu.steer(np.zeros(6), x1)
    n2 = float(np.dot(dp, dp))
    tau_ref = (36.0 * n2) ** 0.25
    assert tau == pytest.approx(tau_ref, rel=1e-14)
    assert J == pytest.approx(4.0 / 3.0 * tau_ref, rel=1e-14)
    assert np.float32(J) == np.float32(4.0 / 3.0 * tau_ref) or \
        abs(np.float32(J) - np.float32(4.0 / 3.0 * tau_ref)) <= np.spacing(np.float32(J))


@pytest.mark.parametrize("v", [[0.5, 0, 0], [0.2, -0.3, 0.4], [1, 1, 1]])
def test_steer_hover_in_place_closed_form(v):
    # same position and velocity v at both ends: tau = 2 sqrt(3) |v|, J = 4 sqrt(3) |v|
    x = np.r_[0.4, 0.4, 0.4, v]
    x1 = x.copy()
    tau, J = cpu.steer(x, x1)
    nv = float(np.linalg.norm(v))
    assert tau == pytest.approx(2 * SQ3 * nv, rel=1e-14)
    assert J == pytest.approx(4 * SQ3 * nv, rel=1e-14)


def test_steer_identical_states_has_no_connection():
    x = np.array([0.3, 0.3, 0.3, 0, 0, 0.0])
    assert cpu.steer(x, x) is None


def _gramian(tau):
    # controllability Gramian of one double-integrator axis by quadrature of e^{As} B B^T e^{A^T s}
    A = np.array([[0.0, 1.0], [0.0, 0.0]])
    B = np.array([[0.0], [1.0]])
    f = lambda s: (scipy.linalg.expm(A * s) @ B @ B.T @ scipy.linalg.expm(A * s).T).ravel()
    return scipy.integrate.quad_vec(f, 0.0, tau, epsabs=0, epsrel=1e-13)[0].reshape(2, 2)


def _J_gramian(x0, x1, tau):
    # time + minimum control energy to reach x1 from x0 in time tau: tau + sum_axes d^T G^-1 d
    A = np.array([[0.0, 1.0], [0.0, 0.0]])
    G = _gramian(tau)
    Ginv = np.linalg.inv(G)
    E = scipy.linalg.expm(A * tau)
    tot = tau
    for j in range(3):
        d = np.array([x1[j], x1[3 + j]]) - E @ np.array([x0[j], x0[3 + j]])
        tot += float(d @ Ginv @ d)
    return tot


def test_steer_matches_gramian_minimum_energy():
    """Cost(u,v) = min_tau [tau + minimum control energy] computed from the controllability
    Gramian (library expm + quadrature) and a bracketed scalar minimiser."""
    rng = np.random.default_rng(11)
    for _ in range(6):
        x0 = np.r_[rng.uniform(0, 1, 3), rng.uniform(-1, 1, 3)]
        x1 = np.r_[rng.uniform(0, 1, 3), rng.uniform(-1, 1, 3)]
        tau, J = cpu.steer(x0, x1)
        grid = np.exp(np.linspace(np.log(0.02), np.log(8.0), 90))
        vals = [_J_gramian(x0, x1, t) for t in grid]
        k = int(np.argmin(vals))
        lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
        res = scipy.optimize.minimize_scalar(lambda t: _J_gramian(x0, x1, t), bounds=(lo, hi),
                                             method="bounded", options={"xatol": 1e-10})
        assert J == pytest.approx(res.fun, rel=1e-8)
        assert J <= res.fun * (1 + 1e-12)
        assert tau == pytest.approx(res.x, rel=1e-3)


def test_steer_root_is_global_minimum_of_J():
    """Dense log-scan plus golden-section refinement of J(tau) never beats the oracle's root."""
    rng = np.random.default_rng(5)
    X0 = np.c_[rng.uniform(0, 1, (300, 3)), rng.uniform(-1, 1, (300, 3))]
    X1 = np.c_[rng.uniform(0, 1, (300, 3)), rng.uniform(-1, 1, (300, 3))]
    grid = np.exp(np.linspace(np.log(1e-3), np.log(50), 4000))
    for x0, x1 in zip(X0, X1):
        dp = x1[:3] - x0[:3]; v0 = x0[3:]; v1 = x1[3:]
        a = v0 @ v0 + v0 @ v1 + v1 @ v1; b = dp @ (v0 + v1); c = dp @ dp
        J = lambda t: t + 4 * a / t - 12 * b / t ** 2 + 12 * c / t ** 3
        vals = J(grid)
        k = int(np.argmin(vals))
        res = scipy.optimize.minimize_scalar(J, bracket=(grid[max(k - 1, 0)], grid[k], grid[min(k + 1, 3999)]),
                                             method="golden", tol=1e-12)
        tau, Jo = cpu.steer(x0, x1)
        assert Jo <= res.fun * (1 + 1e-13)
        assert Jo == pytest.approx(res.fun, rel=1e-12)


def test_steer_two_local_minima_picks_the_lower():
    """Pairs with two local minima of J: the oracle returns the global one."""
    rng = np.random.default_rng(17)
    found = 0
    grid = np.exp(np.linspace(np.log(1e-3), np.log(50), 20000))
    for _ in range(20000):
        x0 = np.r_[rng.uniform(0, 1, 3), rng.uniform(-1, 1, 3)]
        x1 = np.r_[rng.uniform(0, 1, 3), rng.uniform(-1, 1, 3)]
        dp = x1[:3] - x0[:3]; v0 = x0[3:]; v1 = x1[3:]
        a = v0 @ v0 + v0 @ v1 + v1 @ v1; b = dp @ (v0 + v1); c = dp @ dp
        f = grid ** 4 - 4 * a * grid ** 2 + 24 * b * grid - 36 * c
        up = np.nonzero((f[:-1] < 0) & (f[1:] > 0))[0]
        if len(up) < 2:
            continue
        found += 1
        J = grid + 4 * a / grid - 12 * b / grid ** 2 + 12 * c / grid ** 3
        tau, Jo = cpu.steer(x0, x1)
        assert Jo <= J.min() * (1 + 1e-9)
        if found >= 10:
            break
    assert found >= 3


# --------------------------------------------------------------------------- O3
def test_lqr_gain_solves_riccati():
    A = np.array([[0.0, 1.0], [0.0, 0.0]]); B = np.array([[0.0], [1.0]])
    P = scipy.linalg.solve_continuous_are(A, B, np.eye(2), np.eye(1))
    K = (B.T @ P).ravel()
    # the oracle's closed loop A - B K must be A_CL
    assert np.allclose(A - B @ K[None, :], A_CL, atol=1e-14)
    m = cpu.model(0.01, 0.1)
    assert np.allclose(m["Phi"], scipy.linalg.expm(A_CL * 0.1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("sigma", [0.01, 0.3, 1.0])
def test_stationary_covariance_is_lyapunov_solution(sigma):
    m = cpu.model(sigma, 0.05)
    S_ref = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    assert np.allclose(m["S"], S_ref, rtol=1e-13, atol=0)
    assert np.allclose(A_CL @ m["S"] + m["S"] @ A_CL.T + sigma ** 2 * np.eye(2), 0, atol=1e-15 * max(1, sigma ** 2) * 10)
    assert np.allclose(m["Linf"] @ m["Linf"].T, m["S"], rtol=1e-13)


@pytest.mark.parametrize("h", [1e-4, 0.01, 0.1, 0.37, 1.0, 3.0])
def test_transition_and_noise_match_van_loan(h):
    sigma = 0.01
    m = cpu.model(sigma, h)
    assert np.allclose(m["Phi"], scipy.linalg.expm(A_CL * h), rtol=1e-13, atol=1e-16)
    # Van Loan: expm([[-A, V], [0, A^T]] h) gives Q(h) = F22^T F12
    V = sigma ** 2 * np.eye(2)
    M = np.block([[-A_CL, V], [np.zeros((2, 2)), A_CL.T]]) * h
    F = scipy.linalg.expm(M)
    Q_ref = F[2:, 2:].T @ F[:2, 2:]
    # S - Phi S Phi^T cancels for small h: compare against the norm of Q
    assert np.allclose(m["Q"], Q_ref, rtol=0, atol=1e-11 * np.abs(Q_ref).max())
    assert np.all(np.linalg.eigvalsh(m["Q"]) > 0)
    assert np.allclose(m["L"] @ m["L"].T, m["Q"], rtol=1e-12, atol=1e-22)


def test_model_semigroup_and_small_step_limit():
    sigma = 0.2
    a, b = cpu.model(sigma, 0.13), cpu.model(sigma, 0.29)
    ab = cpu.model(sigma, 0.42)
    assert np.allclose(ab["Phi"], a["Phi"] @ b["Phi"], rtol=1e-14, atol=1e-16)
    h = 1e-6
    q = cpu.model(sigma, h)["Q"]
    assert np.allclose(q / h, sigma ** 2 * np.eye(2), rtol=1e-5, atol=1e-9 * sigma ** 2)


# --------------------------------------------------------------------------- O4
def _one_edge_graph(nom, sigma, h, W):
    m = cpu.model(sigma, h)
    return {"n_edges": 1, "W": W, "phi": m["Phi"].astype(np.float32).reshape(1, 4),
            "L": np.array([[m["L"][0, 0], m["L"][1, 0], m["L"][1, 1]]], np.float32),
            "nom": np.asarray(nom, np.float32).reshape(1, W, 3),
            "linf": np.array([m["Linf"][0, 0], m["Linf"][1, 0], m["Linf"][1, 1]], np.float32)}


def test_mask_no_boxes_is_zero_and_cover_all_is_ones():
    W, N = 5, 96
    g = _one_edge_graph(np.full((W, 3), 0.5), 0.01, 0.1, W)
    xi = np.random.default_rng(1).standard_normal((N, W + 1, 3, 2)).astype(np.float32)
    assert np.all(cpu.edge_masks(g, xi, np.zeros((0, 6), np.float32), N) == 0)
    cover = np.array([[-5, -5, -5, 5, 5, 5]], np.float32)
    assert np.all(cpu.edge_masks(g, xi, cover, N) == 0xFFFFFFFF)


def test_mask_zero_noise_equals_nominal_collision():
    W, N = 4, 64
    nom = np.array([[0.1, 0.1, 0.1], [0.3, 0.3, 0.3], [0.5, 0.5, 0.5], [0.7, 0.7, 0.7]])
    xi = np.random.default_rng(2).standard_normal((N, W + 1, 3, 2)).astype(np.float32)
    hit = np.array([[0.45, 0.45, 0.45, 0.55, 0.55, 0.55]], np.float32)
    miss = np.array([[0.8, 0.8, 0.8, 0.9, 0.9, 0.9]], np.float32)
    g = _one_edge_graph(nom, 0.0, 0.1, W)
    assert np.all(cpu.edge_masks(g, xi, hit, N) == 0xFFFFFFFF)
    assert np.all(cpu.edge_masks(g, xi, miss, N) == 0)
    # closed box: a face exactly at the waypoint counts
    face = np.array([[0.5, 0.0, 0.0, 0.6, 1.0, 1.0]], np.float32)
    g2 = _one_edge_graph(np.full((W, 3), np.float32(0.5)), 0.0, 0.1, W)
    assert np.all(cpu.edge_masks(g2, xi, face, N) == 0xFFFFFFFF)


def _bits(masks, N):
    return np.unpackbits(masks.view(np.uint8), bitorder="little")[:N].astype(bool)


def test_mask_single_waypoint_matches_normal_tail():
    """W = 1: the waypoint deviation is stationary N(0, S) (S from scipy's Lyapunov solver), so
    the share of particles beyond a face at distance delta is 1 - Phi(delta / sqrt(S11))."""
    sigma, h, W, N = 0.02, 0.11, 1, 1 << 16
    xi = np.random.default_rng(3).standard_normal((N, W + 1, 3, 2)).astype(np.float32)
    S = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    for k_std in (0.5, 1.0, 2.0):
        delta = k_std * math.sqrt(S[0, 0])
        box = np.array([[0.5 + delta, -1, -1, 3, 3, 3]], np.float32)
        g = _one_edge_graph([[0.5, 0.5, 0.5]], sigma, h, W)
        frac = _bits(cpu.edge_masks(g, xi, box, N), N).mean()
        p = 1 - scipy.stats.norm.cdf(delta / math.sqrt(S[0, 0]))
        assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) / N) + 2e-4


def test_mask_crossing_probability_matches_independent_simulation():
    """W = 10 along a straight line near a face: P(any waypoint beyond the face) depends on the
    step-to-step correlation (Phi, L).  Reference: an independent numpy simulation of the same
    continuous process with scipy expm and Van Loan's integral, fresh normals, 4e5 paths."""
    sigma, h, W, N = 0.02, 0.08, 10, 1 << 16
    S = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    delta = 1.5 * math.sqrt(S[0, 0])
    xi = np.random.default_rng(4).standard_normal((N, W + 1, 3, 2)).astype(np.float32)
    nom = np.c_[np.full(W, 0.5), np.linspace(0.2, 0.8, W), np.full(W, 0.5)]
    box = np.array([[0.5 + delta, -1, -1, 3, 3, 3]], np.float32)
    g = _one_edge_graph(nom, sigma, h, W)
    frac = _bits(cpu.edge_masks(g, xi, box, N), N).mean()
    Phi = scipy.linalg.expm(A_CL * h)
    V = sigma ** 2 * np.eye(2)
    F = scipy.linalg.expm(np.block([[-A_CL, V], [np.zeros((2, 2)), A_CL.T]]) * h)
    Q = F[2:, 2:].T @ F[:2, 2:]
    M = 400000
    rng = np.random.default_rng(99)
    d = rng.multivariate_normal(np.zeros(2), S, size=M)
    hit = np.zeros(M, bool)
    for _ in range(W):
        d = d @ Phi.T + rng.multivariate_normal(np.zeros(2), Q, size=M)
        hit |= d[:, 0] >= delta
    p = hit.mean()
    assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) * (1 / N + 1 / M))


# --------------------------------------------------------------------------- Philox + normals
@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([5, 7, 0, 0], [123, 456]),
                                     ([2 ** 64 - 1, 3, 9, 2 ** 63], [2 ** 64 - 1, 2 ** 40 + 1]),
                                     ([17, 0, 1, 0], [42, 0])])
def test_philox4x64_matches_numpy(ctr, key):
    # numpy's Philox (4x64, 10 rounds) increments the counter before each block
    c = np.array(ctr, dtype=np.uint64)
    prev = c.copy()
    borrow = True
    for i in range(4):
        if not borrow:
            break
        borrow = prev[i] == 0
        prev[i] = np.uint64((int(prev[i]) - 1) % 2 ** 64)
    bg = np.random.Philox(counter=prev, key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4)
    assert np.array_equal(cpu.philox4x64(c, key), ref.astype(np.uint64))


@pytest.mark.parametrize("ctr,key,out", [
    ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1])])
def test_philox4x32_known_answers(ctr, key, out):
    # known-answer vectors published with the generator (Salmon et al., SC'11, Random123)
    assert cpu.philox4x32(ctr, key).tolist() == out


def test_mc_normals_take_the_documented_philox_words():
    # rollout m, step s: one Philox4x32-10 call, counter (m, s lo, 0, s hi), key (seed lo, seed hi);
    # six 21-bit fields: the top 21 bits of each word, then the low 11 bits of word 0 followed by
    # bits 10..1 of word 1, and the same from words 2 and 3; axis j: u1 from field 2j, u2 from
    # field 2j + 1, u = (b + 1/2) / 2^21, Box-Muller in double
    seed, m, s = 0x1234567890ABCDEF, 77, (5 << 32) + 9
    w = np.asarray(cpu.philox4x32([m, s & 0xffffffff, 0, s >> 32], [seed & 0xffffffff, seed >> 32]), np.int64)
    b = [int(w[0]) >> 11, int(w[1]) >> 11, int(w[2]) >> 11, int(w[3]) >> 11,
         ((int(w[0]) & 0x7FF) << 10) | ((int(w[1]) & 0x7FF) >> 1), ((int(w[2]) & 0x7FF) << 10) | ((int(w[3]) & 0x7FF) >> 1)]
    assert all(0 <= x < 2 ** 21 for x in b)
    u = (np.asarray(b, np.float64) + 0.5) / 2.0 ** 21
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    ang = 2.0 * np.pi * u[1::2]
    ref = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1).astype(np.float32)
    np.testing.assert_array_equal(cpu.mc_normals(seed, m, s), ref)


def test_mc_normals_are_standard_normal():
    z = np.concatenate([cpu.mc_normals(7, m, s).ravel() for m in range(300) for s in range(20)])
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.03
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # distinct counters give distinct draws; the same counter repeats
    assert not np.array_equal(cpu.mc_normals(7, 0, 1), cpu.mc_normals(7, 0, 2))
    assert np.array_equal(cpu.mc_normals(7, 3, 4), cpu.mc_normals(7, 3, 4))


# --------------------------------------------------------------------------- O6 MC
def _straight_states(v=0.6, y0=0.2, y1=0.8):
    tau = (y1 - y0) / v
    s0 = np.array([0.5, y0, 0.5, 0.0, v, 0.0], np.float32)
    s1 = np.array([0.5, y1, 0.5, 0.0, v, 0.0], np.float32)
    return np.stack([s0, s1]), np.float32(tau)


def test_mc_no_boxes_and_cover_all():
    st, tau = _straight_states()
    n0 = cpu.mc_certify(st, [0, 1], [tau], 10, 0.01, np.zeros((0, 6), np.float32), 500, 4, 3)
    assert n0 == 0
    n1 = cpu.mc_certify(st, [0, 1], [tau], 10, 0.01, np.array([[-5, -5, -5, 5, 5, 5]], np.float32), 500, 4, 3)
    assert n1 == 500


def test_mc_matches_independent_simulation():
    """Straight constant-velocity connection beside a face: the MC count matches an independent
    simulation of the continuous closed loop sampled at the same 40 sub-steps."""
    sigma, W, S_ = 0.02, 10, 4
    st, tau = _straight_states()
    S = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    delta = 2.0 * math.sqrt(S[0, 0])
    box = np.array([[0.5 + delta, -1, -1, 3, 3, 3]], np.float32)
    M1 = 20000
    c = cpu.mc_certify(st, [0, 1], [tau], W, sigma, box, M1, S_, 11)
    hs = float(np.float32(np.float32(tau / np.float32(W)) / np.float32(S_)))
    Phi = scipy.linalg.expm(A_CL * hs)
    F = scipy.linalg.expm(np.block([[-A_CL, sigma ** 2 * np.eye(2)], [np.zeros((2, 2)), A_CL.T]]) * hs)
    Q = F[2:, 2:].T @ F[:2, 2:]
    M2 = 400000
    rng = np.random.default_rng(5)
    d = rng.multivariate_normal(np.zeros(2), S, size=M2)
    hit = np.zeros(M2, bool)
    for _ in range(W * S_):
        d = d @ Phi.T + rng.multivariate_normal(np.zeros(2), Q, size=M2)
        hit |= d[:, 0] >= delta
    p = hit.mean()
    assert abs(c / M1 - p) <= 5 * math.sqrt(p * (1 - p) * (1 / M1 + 1 / M2))


def _sim_crossing(taus, W, S_, sigma, delta, M, joint, seed):
    """Fraction of closed-loop deviation paths whose x component reaches delta at some sub-step of
    a path of connections with durations `taus` (independent numpy simulation: exact transition
    e^{A h} and Van Loan noise per step, h = float(float(tau / W) / substeps)).  joint: 'carry'
    keeps the deviation through each joint, 'redraw' draws it afresh from the stationary law,
    'zero' resets it to 0."""
    S = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    rng = np.random.default_rng(seed)
    d = rng.multivariate_normal(np.zeros(2), S, size=M)
    hit = np.zeros(M, bool)
    for ei, tau in enumerate(taus):
        if ei > 0 and joint == "redraw":
            d = rng.multivariate_normal(np.zeros(2), S, size=M)
        elif ei > 0 and joint == "zero":
            d = np.zeros((M, 2))
        hs = float(np.float32(np.float32(np.float32(tau) / np.float32(W)) / np.float32(S_)))
        Phi = scipy.linalg.expm(A_CL * hs)
        F = scipy.linalg.expm(np.block([[-A_CL, sigma ** 2 * np.eye(2)], [np.zeros((2, 2)), A_CL.T]]) * hs)
        Q = F[2:, 2:].T @ F[:2, 2:]
        for _ in range(W * S_):
            d = d @ Phi.T + rng.multivariate_normal(np.zeros(2), Q, size=M)
            hit |= d[:, 0] >= delta
    return float(hit.mean())


def test_mc_carries_deviation_across_connections():
    """MC(p) (Section III-A) is the collision probability of the whole plan: the tracking
    deviation runs on through the joint between two connections.  Two straight constant-velocity
    connections of different durations (so different sub-step sizes) beside a face: the oracle's
    count matches an independent simulation that carries the deviation through the joint, and is
    far from what re-drawing it at the joint or resetting it to zero would give (about 27 and 14
    standard errors apart), so either mistake in the oracle fails here."""
    sigma, W, S_, v = 0.02, 10, 4, 0.6
    taus = [np.float32(0.15), np.float32(0.35)]
    ys = [0.2, 0.2 + 0.6 * 0.15, 0.2 + 0.6 * 0.5]
    st = np.array([[0.5, y, 0.5, 0.0, v, 0.0] for y in ys], np.float32)
    S = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    delta = 1.5 * math.sqrt(S[0, 0])
    box = np.array([[0.5 + delta, -1, -1, 3, 3, 3]], np.float32)
    M1, M2 = 20000, 200000
    c = cpu.mc_certify(st, [0, 1, 2], taus, W, sigma, box, M1, S_, 17)
    p_carry = _sim_crossing(taus, W, S_, sigma, delta, M2, "carry", 5)
    sd = math.sqrt(p_carry * (1 - p_carry) * (1 / M1 + 1 / M2))
    assert abs(c / M1 - p_carry) <= 5 * sd, (c / M1, p_carry, sd)
    for joint in ("redraw", "zero"):
        p_alt = _sim_crossing(taus, W, S_, sigma, delta, M2, joint, 6)
        assert abs(c / M1 - p_alt) > 8 * sd, (joint, c / M1, p_alt, sd)


# --------------------------------------------------------------------------- thresholds
def test_cp_thresholds_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "cp_thresholds.txt")) if l.strip() and not l.startswith("#")]
    for a, e, n, kmin, kmax in rows:
        assert cpu.cp_thresholds(float(a), float(e), int(n)) == (int(kmin), int(kmax))


# --------------------------------------------------------------------------- O2 graph
def test_graph_pruning_shortcut_is_exact():
    wl = inputs.make_workload("three_box_1k", seed=3, n_samples=120)
    a = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma, exhaustive=False)
    b = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma, exhaustive=True)
    for k in ("row_ptr", "col", "ecost", "tau", "phi", "L", "nom"):
        assert np.array_equal(a[k], b[k]), k
    assert a["pairs_costed"] < b["pairs_costed"]


def test_graph_edges_are_the_cost_ball_without_collisions():
    """Neighbour sets equal {u : float(Cost(v,u)) < r} by brute force over all pairs, minus the
    pairs whose connection hits a box at the 4W check times t_m = m tau / (4W).  The check
    positions are evaluated independently with scipy's cubic Hermite interpolant of the end
    states (the minimum-effort connection for a fixed duration)."""
    wl = inputs.make_workload("three_box_1k", seed=1, n_samples=60)
    W = wl.n_waypoints
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, W, wl.sigma)
    st = wl.states.astype(np.float64)
    n = st.shape[0]
    inside = lambda p: np.any(np.all((wl.boxes[None, :, :3] <= p[:, None, :]) &
                                     (p[:, None, :] <= wl.boxes[None, :, 3:]), axis=2), axis=1)
    n_dropped = 0
    for v in range(n):
        nbrs = set(g["col"][g["row_ptr"][v]:g["row_ptr"][v + 1]].tolist())
        if inside(wl.states[v:v + 1, :3])[0]:
            assert not nbrs
            continue
        for u in range(n):
            if u == v or inside(wl.states[u:u + 1, :3])[0]:
                assert u not in nbrs
                continue
            tj = cpu.steer(st[v], st[u])
            if not np.float32(tj[1]) < np.float32(wl.radius):
                assert u not in nbrs
                continue
            tau = float(np.float32(tj[0]))
            ts = tau * (np.arange(1, 4 * W + 1) / (4 * W))
            p = np.stack([scipy.interpolate.CubicHermiteSpline([0, tau], [st[v, j], st[u, j]],
                                                               [st[v, 3 + j], st[u, 3 + j]])(ts)
                          for j in range(3)], axis=1).astype(np.float32)
            hit = bool(inside(p).any())
            assert (u in nbrs) == (not hit), (v, u)
            n_dropped += hit
    assert n_dropped > 0


def test_nominal_waypoints_follow_hermite_cubic():
    """The min-effort connection for fixed duration is the cubic Hermite interpolant of the end
    states; the oracle's waypoints at t_k = k h equal scipy's interpolant there."""
    wl = inputs.make_workload("three_box_1k", seed=2, n_samples=40)
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    st = wl.states.astype(np.float64)
    W = wl.n_waypoints
    for v in range(g["n"]):
        for e in range(g["row_ptr"][v], g["row_ptr"][v + 1]):
            u = g["col"][e]
            tau = float(g["tau"][e]); h = float(g["h"][e])
            assert np.float32(h) == np.float32(np.float32(tau) / np.float32(W))
            for j in range(3):
                sp = scipy.interpolate.CubicHermiteSpline([0, tau], [st[v, j], st[u, j]], [st[v, 3 + j], st[u, 3 + j]])
                ref = sp(np.arange(1, W + 1) * h)
                assert np.allclose(g["nom"][e, :, j], ref, rtol=0, atol=4e-7)


# --------------------------------------------------------------------------- O5 Explore
def _dijkstra_f32(n, row_ptr, col, ecost, s):
    import heapq
    dist = [None] * n
    dist[s] = np.float32(0)
    pq = [(0.0, s)]
    done = [False] * n
    while pq:
        d, v = heapq.heappop(pq)
        if done[v]:
            continue
        done[v] = True
        for e in range(row_ptr[v], row_ptr[v + 1]):
            u = int(col[e])
            nd = np.float32(dist[v] + np.float32(ecost[e]))
            if dist[u] is None or nd < dist[u]:
                dist[u] = nd
                heapq.heappush(pq, (float(nd), u))
    return dist


@pytest.mark.parametrize("seed", range(4))
def test_explore_zero_masks_equals_dijkstra(seed):
    g = inputs.random_explore_graph(300, 12, 32, seed, bit_prob=0.0, hot_edge_frac=0.0)
    ex = cpu.explore(g.n, g.row_ptr, g.col, g.ecost, g.emask, 0, [1], 1, 4, 0.5, g.radius,
                     flags=cpu.NO_EARLY_STOP)
    assert ex["status"] == cpu.OK
    dist = _dijkstra_f32(g.n, g.row_ptr, g.col, g.ecost, 0)
    best = {}
    for p in range(ex["n_plans"]):
        if ex["removed"][p]:
            continue
        x = int(ex["head"][p])
        best[x] = min(best.get(x, np.float32(np.inf)), ex["cost"][p])
    reach = [v for v in range(g.n) if dist[v] is not None]
    assert set(best) == set(reach)
    for v in reach:
        assert best[v] == dist[v]


def _tiny_graph(seed, n):
    rng = np.random.default_rng(seed)
    rows, cols, costs, masks = [0], [], [], []
    for v in range(n):
        nb = sorted(rng.choice([u for u in range(n) if u != v], size=rng.integers(0, n), replace=False).tolist())
        cols += nb
        costs += rng.uniform(0.3, 1.0, len(nb)).astype(np.float32).tolist()
        masks += (rng.random(len(nb)) < 0.35).astype(np.uint32).tolist()
        rows.append(len(cols))
    return (np.asarray(rows, np.int32), np.asarray(cols, np.int32), np.asarray(costs, np.float32),
            np.asarray(masks, np.uint32).reshape(-1, 1))


def _pareto(values):
    vals = set(values)
    return {v for v in vals if not any((w[0] <= v[0] and w[1] <= v[1]) and w != v for w in vals)}


@pytest.mark.parametrize("seed", range(12))
def test_explore_single_particle_equals_bruteforce_pareto_front(seed):
    """One particle bit, no CP cutoff, no early stop: the non-dominated (cost, bit) values among
    the plans left at each node equal the Pareto front over all simple paths from the start."""
    n = 6
    rp, col, ec, em = _tiny_graph(seed, n)
    ex = cpu.explore(n, rp, col, ec, em, 0, [n - 1], 1, 2, 0.5, 1.0, flags=cpu.NO_EARLY_STOP)
    assert ex["status"] == cpu.OK
    paths = {v: [] for v in range(n)}

    def dfs(v, visited, cost, bit):
        paths[v].append((np.float32(cost), bit))
        for e in range(rp[v], rp[v + 1]):
            u = int(col[e])
            if u in visited:
                continue
            dfs(u, visited | {u}, np.float32(np.float32(cost) + ec[e]), bit | int(em[e, 0] & 1))

    dfs(0, {0}, np.float32(0), 0)
    for v in range(n):
        live = [(ex["cost"][p], int(ex["popc"][p])) for p in range(ex["n_plans"])
                if not ex["removed"][p] and ex["head"][p] == v]
        assert _pareto(live) == _pareto(paths[v]), v


@pytest.mark.parametrize("seed,n,deg,N,kmax,early", [(0, 40, 5, 32, 3, False), (1, 40, 6, 64, 4, True),
                                                    (2, 60, 4, 32, 2, True), (3, 30, 8, 32, 33, False),
                                                    (4, 50, 5, 64, 6, False), (5, 25, 6, 32, 1, False)])
def test_explore_matches_naive_restatement(seed, n, deg, N, kmax, early):
    g = inputs.random_explore_graph(n, deg, N, seed, radius=1.0, bit_prob=0.05, hot_edge_frac=0.2,
                                    hot_bit_prob=0.3)
    goal = [n - 1, n - 2]
    flags = 0 if early else cpu.NO_EARLY_STOP
    a = cpu.explore(g.n, g.row_ptr, g.col, g.ecost, g.emask, 0, goal, 1, kmax, 0.5, g.radius, flags=flags)
    b = naive.explore_naive(g.n, g.row_ptr, g.col, g.ecost, g.emask, 0, goal, 1, kmax, 0.5, g.radius,
                            no_early_stop=not early)
    assert a["n_plans"] == b["n_plans"]
    for k in ("head", "parent", "cost", "popc", "t_created", "e_expanded", "removed", "goal_plans"):
        assert np.array_equal(a[k], b[k]), k
    mi = [sum(int(a["mask"][p, j]) << (32 * j) for j in range(g.n_words)) for p in range(a["n_plans"])]
    assert mi == b["mask_int"]
    assert a["n_candidates"] == b["n_candidates"]
    assert a["n_iterations"] == b["n_iterations"]


def test_explore_invariants_on_dynamics_graph():
    wl = inputs.make_workload("three_box_1k", seed=0, n_samples=200)
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    masks = cpu.edge_masks(g, wl.xi, wl.boxes, wl.n_particles)
    kmin, kmax = cpu.cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    ex = cpu.explore(g["n"], g["row_ptr"], g["col"], g["ecost"], masks, 0, wl.goal_idx, kmin, kmax, wl.lam,
                     wl.radius)
    assert ex["status"] == cpu.OK and ex["n_plans"] > 1
    for p in range(1, ex["n_plans"]):
        path = cpu.backtrack(ex["parent"], ex["head"], p)
        c = np.float32(0); m = np.zeros(masks.shape[1], np.uint32)
        for k in range(len(path) - 1):
            e = cpu.edge_of(g, int(path[k]), int(path[k + 1]))
            c = np.float32(c + g["ecost"][e]); m |= masks[e]
        assert ex["cost"][p] == c
        assert np.array_equal(ex["mask"][p], m)
        assert ex["popc"][p] == sum(bin(int(x)).count("1") for x in m) < kmax
    # no live open plan is dominated at its head
    for p in range(ex["n_plans"]):
        if ex["removed"][p] or ex["e_expanded"][p] >= 0:
            continue
        same = [q for q in range(ex["n_plans"]) if not ex["removed"][q] and ex["head"][q] == ex["head"][p]]
        assert not any(ex["cost"][q] < ex["cost"][p] and ex["popc"][q] <= ex["popc"][p] for q in same)


def test_explore_start_in_goal_stops_immediately():
    g = inputs.random_explore_graph(20, 4, 32, 0)
    ex = cpu.explore(g.n, g.row_ptr, g.col, g.ecost, g.emask, 3, [3], 1, 3, 0.5, g.radius)
    assert ex["n_plans"] == 1 and ex["n_candidates"] == 0 and list(ex["goal_plans"]) == [0]


def test_explore_capacity_error():
    g = inputs.random_explore_graph(200, 10, 32, 1)
    ex = cpu.explore(g.n, g.row_ptr, g.col, g.ecost, g.emask, 0, [1], 1, 3, 0.5, g.radius, max_plans=50,
                     flags=cpu.NO_EARLY_STOP)
    assert ex["status"] == cpu.ERR_CAPACITY


# --------------------------------------------------------------------------- all-cores oracle
@pytest.mark.parametrize("threads", [2, 5])
def test_all_cores_oracle_equals_single_thread(threads):
    """The threaded oracle (used only to time the oracle on every host core) gives the
    single-thread masks and Explore result exactly."""
    wl = inputs.make_workload("indoor_4k", seed=1, n_samples=500)
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    m1 = cpu.edge_masks(g, wl.xi, wl.boxes, wl.n_particles)
    mt = cpu.edge_masks(g, wl.xi, wl.boxes, wl.n_particles, n_threads=threads)
    assert np.array_equal(m1, mt) and m1.any()
    kmin, kmax = cpu.cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    for flags in (0, cpu.NO_EARLY_STOP):
        a = cpu.explore(g["n"], g["row_ptr"], g["col"], g["ecost"], m1, 0, wl.goal_idx, kmin, kmax, wl.lam,
                        wl.radius, flags=flags)
        b = cpu.explore(g["n"], g["row_ptr"], g["col"], g["ecost"], m1, 0, wl.goal_idx, kmin, kmax, wl.lam,
                        wl.radius, flags=flags, n_threads=threads)
        for k in ("status", "n_plans", "n_candidates", "n_kept", "n_iterations", "n_groups_expanded", "n_goal"):
            assert a[k] == b[k], k
        for k in ("head", "parent", "mask", "popc", "t_created", "e_expanded", "removed", "goal_plans"):
            assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a["cost"].view(np.uint32), b["cost"].view(np.uint32))
