"""Pins of the oracle's Half-Space Monte Carlo (HSMC) masks (section 'Half-Space Monte Carlo',
Eq. (eq:hs)) against what the construction must give: closed-form half-spaces for single boxes at
perpendicular, parallel and oblique travel; boxes hidden behind a nearer one pruned; on random
scenes, the first half-space at the true nearest obstacle point (found by dense sampling of the
boxes) and every pruned box inside its half-space (checked at its eight corners); the region
capped at hmax; and the firing rate of particles at one waypoint equal to the normal tail
1 - Phi(|a| / sqrt(S11)) (S from scipy's Lyapunov solver)."""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from oracle import cpu

A_CL = np.array([[0.0, 1.0], [-1.0, -math.sqrt(3.0)]])
Y = np.array([0.5, 0.5, 0.5], np.float32)
NEAR = [0.6, 0.4, 0.4, 0.7, 0.6, 0.6]   # +x, closest point (0.6, 0.5, 0.5)
HIDDEN = [0.8, 0.4, 0.4, 0.9, 0.6, 0.6]  # behind NEAR
OPPOSITE = [0.2, 0.45, 0.45, 0.3, 0.55, 0.55]  # -x, closest point (0.3, 0.5, 0.5)


def test_single_box_perpendicular_motion_gives_the_separating_plane():
    a, b = cpu.halfspaces(Y, [0, 1, 0], [NEAR])
    assert a.shape == (1, 3)
    np.testing.assert_allclose(a[0], [0.1, 0, 0], atol=1e-7)
    assert b[0] == pytest.approx(0.01, rel=1e-6)


def test_motion_along_the_obstacle_direction_removes_the_constraint():
    a, b = cpu.halfspaces(Y, [2.0, 0, 0], [NEAR])
    np.testing.assert_array_equal(a[0], [0, 0, 0])
    assert b[0] == 0


def test_oblique_motion_projects_out_the_travel_direction():
    # d = (0.1, 0, 0), v = (1, 1, 0): a = d - (d.v / v.v) v = (0.05, -0.05, 0), b = 0.005
    a, b = cpu.halfspaces(Y, [1, 1, 0], [NEAR])
    np.testing.assert_allclose(a[0], [0.05, -0.05, 0], atol=1e-7)
    assert b[0] == pytest.approx(0.005, rel=1e-5)
    assert abs(float(np.dot(a[0], [1, 1, 0]))) < 1e-7   # a is perpendicular to the motion


def test_hidden_box_is_pruned_and_opposite_box_kept():
    a, b = cpu.halfspaces(Y, [0, 0, 1], [HIDDEN, NEAR, OPPOSITE])
    assert len(b) == 2
    np.testing.assert_allclose(a, [[0.1, 0, 0], [-0.2, 0, 0]], atol=1e-6)
    assert b[0] <= b[1]


def test_zero_velocity_uses_the_distance_vector():
    a, b = cpu.halfspaces(Y, [0, 0, 0], [OPPOSITE])
    np.testing.assert_allclose(a[0], [-0.2, 0, 0], atol=1e-6)


def test_region_capped_at_hmax():
    boxes = []
    for k in range(12):
        ang = 2 * math.pi * k / 12
        c = 0.5 + 0.3 * np.array([math.cos(ang), math.sin(ang), 0.0])
        boxes.append([c[0] - 0.02, c[1] - 0.02, 0.45, c[0] + 0.02, c[1] + 0.02, 0.55])
    a_full, _ = cpu.halfspaces(Y, [0, 0, 1], boxes, hmax=32)
    a_cap, _ = cpu.halfspaces(Y, [0, 0, 1], boxes, hmax=5)
    assert len(a_full) == 12 and len(a_cap) == 5
    np.testing.assert_array_equal(a_cap, a_full[:5])


@pytest.mark.parametrize("seed", range(6))
def test_random_scene_regions_follow_the_construction(seed):
    """v = 0 (a = d): each d points at the nearest point of the nearest box still in play; boxes
    pruned at a step lie in {z : d.(z - y) >= d.d}; distances never decrease."""
    g = np.random.default_rng(100 + seed)
    nb = 9
    lo = g.uniform(0.0, 0.9, size=(nb, 3))
    boxes = np.concatenate([lo, lo + g.uniform(0.03, 0.15, size=(nb, 3))], axis=1).astype(np.float32)
    y = g.uniform(0.0, 1.0, size=3).astype(np.float32)
    inside = np.all((boxes[:, :3] <= y) & (y <= boxes[:, 3:]), axis=1)
    if inside.any():
        pytest.skip("waypoint inside a box")
    a, b = cpu.halfspaces(y, [0, 0, 0], boxes, hmax=64)
    # dense samples of every box (float64) give its distance to y independently of the clamp formula
    t = np.linspace(0.0, 1.0, 41)
    grid = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    dist = np.array([np.min(np.linalg.norm(bx[:3] + grid * (bx[3:] - bx[:3]) - y, axis=1)) for bx in boxes.astype(np.float64)])
    remaining = set(range(nb))
    prev = -1.0
    for d, bb in zip(a.astype(np.float64), b):
        r = math.sqrt(float(np.dot(d, d)))
        nearest = min(remaining, key=lambda o: dist[o])
        assert r <= dist[nearest] + 1e-6 and r >= dist[nearest] - 0.02   # grid spacing bound
        assert r >= prev - 1e-7
        prev = r
        corners = np.array([[bx[0 if i & 1 == 0 else 3], bx[1 if i & 2 == 0 else 4], bx[2 if i & 4 == 0 else 5]]
                            for bx in boxes.astype(np.float64) for i in range(8)]).reshape(nb, 8, 3)
        inside_hs = np.all((corners - y) @ d >= np.dot(d, d) - 1e-6, axis=1)
        pruned = {o for o in remaining if inside_hs[o]}
        assert nearest in pruned or r > dist[nearest] - 1e-6
        remaining -= pruned | {nearest}
    assert not remaining   # every box pruned (hmax not reached)


def _bits(masks, N):
    return np.unpackbits(masks.view(np.uint8), bitorder="little")[:N].astype(bool)


def _one_edge(y, v, sigma, h):
    m = cpu.model(sigma, h)
    return {"n_edges": 1, "W": 1, "phi": m["Phi"].astype(np.float32).reshape(1, 4),
            "L": np.array([[m["L"][0, 0], m["L"][1, 0], m["L"][1, 1]]], np.float32),
            "nom": np.asarray(y, np.float32).reshape(1, 1, 3), "nvel": np.asarray(v, np.float32).reshape(1, 1, 3),
            "linf": np.array([m["Linf"][0, 0], m["Linf"][1, 0], m["Linf"][1, 1]], np.float32)}


def test_no_boxes_or_no_noise_never_fires():
    xi = np.random.default_rng(4).standard_normal((64, 2, 3, 2)).astype(np.float32)
    g = _one_edge(Y, [0, 1, 0], 0.02, 0.1)
    assert not cpu.edge_masks_hs(g, xi, np.zeros((0, 6), np.float32), 64).any()
    g0 = _one_edge(Y, [0, 1, 0], 0.0, 0.1)
    assert not cpu.edge_masks_hs(g0, xi, np.array([NEAR], np.float32), 64).any()


@pytest.mark.parametrize("k_std", [0.5, 1.0, 2.0])
def test_firing_rate_matches_normal_tail(k_std):
    """One waypoint, one box at distance |a| = k sqrt(S11) across the travel direction: the
    deviation is stationary N(0, S11 I) in position, so a.dy ~ N(0, S11 |a|^2) and the share of
    firing particles is 1 - Phi(|a| / sqrt(S11))."""
    sigma, h, N = 0.02, 0.11, 1 << 15
    S = scipy.linalg.solve_continuous_lyapunov(A_CL, -sigma ** 2 * np.eye(2))
    delta = k_std * math.sqrt(S[0, 0])
    box = np.array([[0.5 + delta, 0.0, 0.0, 1.0, 1.0, 1.0]], np.float32)
    xi = np.random.default_rng(5).standard_normal((N, 2, 3, 2)).astype(np.float32)
    frac = _bits(cpu.edge_masks_hs(_one_edge(Y, [0, 1, 0], sigma, h), xi, box, N), N).mean()
    p = 1 - scipy.stats.norm.cdf(delta / math.sqrt(S[0, 0]))
    assert abs(frac - p) <= 5 * math.sqrt(p * (1 - p) / N) + 3e-4
