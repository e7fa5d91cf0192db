"""Pins of the dense PnP + RANSAC oracle (Sec. 3.4, Eq. 10): the P3P solver
against exact synthetic views, lifting against projection, RANSAC against a
planted inlier set, Gauss-Newton against the stationarity of its cost; no GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import pnp
from paper_2507_15683_gb300 import synth

CAM = {"width": 640, "height": 480, "fx": 500.0, "fy": 520.0, "cx": 321.0, "cy": 239.0}


def _pose(g):
    T = synth.perturb_pose(np.eye(4), g, 40.0, 0.0)
    T[:3, 3] = g.normal(0, 20, 3)
    return T


def _points_in_view(g, T, n, zmin=30.0, zmax=400.0):
    """World points whose camera-frame depth is in [zmin, zmax] and that project
    inside the image; returns X (n, 3) and exact pixel positions (n, 2)."""
    fx, fy, cx, cy = (float(np.float32(CAM[k])) for k in ("fx", "fy", "cx", "cy"))
    u = g.uniform(0, CAM["width"], n)
    v = g.uniform(0, CAM["height"], n)
    z = g.uniform(zmin, zmax, n)
    pc = np.stack([(u - cx) / fx * z, (v - cy) / fy * z, z], 1)
    X = (pc - T[:3, 3]) @ T[:3, :3]
    return X, np.stack([u, v], 1)


def _rot_deg(Ra, Rb):
    c = np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1)
    return math.degrees(math.acos(c))


def test_p3p_recovers_the_true_pose():
    g = np.random.default_rng(0)
    found, n_near = 0, 0
    for trial in range(200):
        T = _pose(g)
        X, px = _points_in_view(g, T, 3)
        f = pnp.bearings(px, CAM)
        sols, near = pnp.p3p(X, f)
        assert len(sols) <= 4
        for R, t, v in sols:
            assert np.allclose(R @ R.T, np.eye(3), atol=1e-9) and np.linalg.det(R) == pytest.approx(1.0, abs=1e-9)
            # every solution reprojects the three points exactly
            e, _ = pnp.reproj_err(R, t, X, px, CAM)
            assert np.all(e < 1e-3), e  # rounding in ill-conditioned triangles stays below 3e-4 px
        best = min((_rot_deg(R, T[:3, :3]) + np.linalg.norm(t - T[:3, 3]) for R, t, _ in sols), default=np.inf)
        if near:
            n_near += 1
            continue
        assert best < 1e-4, (trial, best, len(sols))  # degrees + metres; a wrong root or frame is off by O(1)
        found += 1
    assert found >= 190


def test_quartic_vanishes_at_the_true_distance_ratio():
    g = np.random.default_rng(1)
    for _ in range(50):
        T = _pose(g)
        X, px = _points_in_view(g, T, 3)
        f = pnp.bearings(px, CAM)
        Q, _ = pnp.quartic(X, f)
        s = np.linalg.norm(X @ T[:3, :3].T + T[:3, 3], axis=1)  # true distances along the rays
        v = s[2] / s[0]
        scale = np.sum(np.abs(Q) * np.maximum(1.0, v) ** np.arange(5))
        assert abs(np.polynomial.polynomial.polyval(v, Q)) < 1e-12 * scale


def test_lift_projects_back_to_the_rendered_pixel():
    g = np.random.default_rng(2)
    T = _pose(g)
    H, W = CAM["height"], CAM["width"]
    alpha = g.uniform(0.3, 1.0, (H, W))
    z = g.uniform(50, 300, (H, W))
    depth = alpha * z
    r = g.choice(H * W, 500, replace=False)
    q = g.choice(H * W, 500, replace=False)
    m = np.stack([np.zeros(500, np.int64), q, r], 1)
    X, p, valid = pnp.lift(depth, alpha, CAM, T, m)
    np.testing.assert_array_equal(valid, alpha.reshape(-1)[r] >= 0.5)
    rp = np.stack([(r % W) + 0.5, (r // W) + 0.5], 1)
    e, pc = pnp.reproj_err(T[:3, :3], T[:3, 3], X[valid], rp[valid], CAM)
    assert np.all(e < 1e-8)
    np.testing.assert_allclose(pc[:, 2], z.reshape(-1)[r][valid], rtol=1e-12)
    np.testing.assert_array_equal(p, np.stack([(q % W) + 0.5, (q // W) + 0.5], 1))


def test_sample_indices_are_floor_of_scaled_words():
    g = np.random.default_rng(3)
    w = g.integers(0, 2 ** 32, (100, 3), dtype=np.uint64)
    for K in (1, 3, 7, 1000, 2_000_003):
        idx = pnp.sample_indices(w, K)
        for a, b in zip(w.reshape(-1).tolist(), idx.reshape(-1).tolist()):
            assert b == (a * K) // (2 ** 32)
            assert 0 <= b < K


def _planted(g, n=1500, out_frac=0.3, noise=0.0):
    T = _pose(g)
    X, px = _points_in_view(g, T, n)
    n_out = int(n * out_frac)
    px = px + g.normal(0, noise, px.shape) if noise else px.copy()
    px[:n_out] = np.stack([g.uniform(0, CAM["width"], n_out), g.uniform(0, CAM["height"], n_out)], 1)
    return T, X, px, n_out


def test_ransac_finds_the_planted_pose_and_inliers():
    g = np.random.default_rng(4)
    T, X, px, n_out = _planted(g)
    words = g.integers(0, 2 ** 32, (64, 3), dtype=np.uint64)
    rs = pnp.ransac(X, px, CAM, words, tau=2.0)
    h, s = rs["best"]
    R, t, _ = rs["hyps"][h][s]
    assert _rot_deg(R, T[:3, :3]) < 1e-6 and np.linalg.norm(t - T[:3, 3]) < 1e-6
    e_true, _ = pnp.reproj_err(T[:3, :3], T[:3, 3], X, px, CAM)
    assert rs["best_count"] == int((e_true < 2.0).sum())
    # the best is the first maximum over (hypothesis, solution)
    flat = [(c, -hh, -ss) for hh, cs in enumerate(rs["counts"]) for ss, c in enumerate(cs)]
    assert max(flat) == (rs["best_count"], -h, -s)


def test_gauss_newton_reaches_a_stationary_point_of_the_inlier_cost():
    g = np.random.default_rng(5)
    T, X, px, n_out = _planted(g, noise=0.6)
    T0 = O.se3_exp_left(np.r_[g.normal(0, 0.3, 3), g.normal(0, 0.002, 3)], T)
    Tf, hist = pnp.gn_refine(T0, X, px, CAM, 3.0, 12)
    inl, _ = pnp.inliers(Tf[:3, :3], Tf[:3, 3], X, px, CAM, 3.0)
    assert inl.sum() > 0.6 * len(X)

    def cost(xi):
        Tx = O.se3_exp_left(xi, Tf)
        e, _ = pnp.reproj_err(Tx[:3, :3], Tx[:3, 3], X[inl], px[inl], CAM)
        return float(np.sum(e ** 2))

    c0 = cost(np.zeros(6))
    for k, h in enumerate([1e-4] * 3 + [1e-6] * 3):
        d = np.zeros(6)
        d[k] = h
        grad = (cost(d) - cost(-d)) / (2 * h)
        curv = (cost(d) - 2 * c0 + cost(-d)) / (h * h)
        assert abs(grad) <= 1e-6 * curv * (1 if k < 3 else 1e-2) + 1e-7 * c0, (k, grad, curv)
    # the noise-free planted pose is recovered exactly
    T2, X2, px2, _ = _planted(np.random.default_rng(6))
    T20 = O.se3_exp_left(np.r_[0.5, -0.3, 0.2, 0.003, -0.002, 0.001], T2)
    Tf2, _ = pnp.gn_refine(T20, X2, px2, CAM, 3.0, 10)
    assert _rot_deg(Tf2[:3, :3], T2[:3, :3]) < 1e-7 and np.linalg.norm(Tf2[:3, 3] - T2[:3, 3]) < 1e-6
