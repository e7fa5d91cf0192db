"""Pins of the oracle's colour (SH) and compositing layers.

Sec. 3.1 of the paper: colours are alpha-blended by the rasterizer, features
go through the identical blending. The blending constants (alpha floor 1/255,
cap 0.99, transmittance cutoff 1e-4 with stop-before-blend, background 0,
depth = sum of w z) are this project's readings; the expected values below are
closed forms of those rules, invariants, or a brute-force walk.
"""
import math

import numpy as np
import pytest

from paper_2507_15683_gb300 import synth
from tests.oracle_scenes import Y00, cam, scene_of


# --------------------------------------------------------------------------
# spherical harmonics
# --------------------------------------------------------------------------

def _sphere_quadrature(n_theta=24, n_phi=48):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # cos(theta) nodes
    phis = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    pts, wts = [], []
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            pts.append((st * math.cos(ph), st * math.sin(ph), ct))
            wts.append(wt * 2 * math.pi / n_phi)
    return np.array(pts), np.array(wts)


def test_sh_orthonormal_by_quadrature(oracle):
    pts, wts = _sphere_quadrature()
    Y = np.stack([oracle.sh_basis(3, p)[0] for p in pts])
    G = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_addition_theorem(oracle):
    # sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b)
    g = np.random.default_rng(1)
    P = [lambda t: 1.0, lambda t: t, lambda t: 0.5 * (3 * t * t - 1), lambda t: 0.5 * (5 * t ** 3 - 3 * t)]
    for _ in range(20):
        a, b = g.standard_normal(3), g.standard_normal(3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        Ya, Yb = oracle.sh_basis(3, a)[0], oracle.sh_basis(3, b)[0]
        for l in range(4):
            sl = slice(l * l, (l + 1) ** 2)
            assert np.dot(Ya[sl], Yb[sl]) == pytest.approx((2 * l + 1) / (4 * math.pi) * P[l](a @ b), abs=1e-13)


def test_sh_degree0_and_1_convention(oracle):
    d = np.array([0.36, -0.48, 0.8])
    Y, _ = oracle.sh_basis(1, d)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y, [Y00, -c1 * d[1], c1 * d[2], -c1 * d[0]], rtol=1e-14)


def test_sh_gradient_matches_finite_differences(oracle):
    g = np.random.default_rng(2)
    for _ in range(10):
        d = g.standard_normal(3)
        _, dY = oracle.sh_basis(3, d)
        h = 1e-6
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / (2 * h)
            np.testing.assert_allclose(dY[:, k], fd, atol=1e-8)


# --------------------------------------------------------------------------
# compositing closed forms
# --------------------------------------------------------------------------

def F32(x):
    """The binary32 value of an input parameter, as a binary64 number."""
    return float(np.float32(x))


def _pix_centres(c):
    ys, xs = np.mgrid[0:c["height"], 0:c["width"]]
    return xs.ravel() + 0.5, ys.ravel() + 0.5


def _tile_mask(c, x0, x1, y0, y1):
    xs, ys = _pix_centres(c)
    tx, ty = (xs // 16).astype(int), (ys // 16).astype(int)
    return (tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)


def _single_alpha(c, u, v, var, o):
    xs, ys = _pix_centres(c)
    power = -0.5 * ((u - xs) ** 2 + (v - ys) ** 2) / var
    a = np.minimum(0.99, o * np.exp(power))
    return np.where(a < 1 / 255, 0.0, a)


def test_single_gaussian_closed_form(oracle):
    # isotropic s = 0.1 at z = 5 on the axis: Sigma' = 4.3 I, tiles 3..4 (see projection pins)
    dc = np.array([[0.3, -0.2, 0.9]], np.float32)
    sc = scene_of([[0, 0, 5]], [[0.1] * 3], opacities=[0.8], dc=dc)
    c = cam()
    r = oracle.render(sc, c, np.eye(4), geom64=True)
    rgb = 0.5 + Y00 * dc[0].astype(np.float64)
    var = (100 * F32(0.1) / 5) ** 2 + 0.3
    a = _single_alpha(c, 64.0, 64.0, var, F32(0.8)) * _tile_mask(c, 3, 4, 3, 4)
    np.testing.assert_allclose(r["alpha"], a, atol=1e-12)
    np.testing.assert_allclose(r["rgb"], a[:, None] * rgb[None, :], atol=1e-12)
    np.testing.assert_allclose(r["depth"], 5.0 * a, atol=1e-12)
    assert r["alpha"].max() > 0.7 and (r["alpha"] == 0).sum() > 0


def test_two_stacked_gaussians(oracle):
    # C = a1 c1 + (1 - a1) a2 c2 for a front Gaussian at z = 5 and a back one at z = 6
    dc = np.array([[0.4, 0.1, -0.3], [-0.2, 0.6, 0.2]], np.float32)
    sc = scene_of([[0, 0, 6], [0, 0, 5]], [[0.1] * 3, [0.12] * 3], opacities=[0.7, 0.6], dc=dc[::-1].copy())
    c = cam()
    r = oracle.render(sc, c, np.eye(4), geom64=True)
    o = np.float32([0.7, 0.6]).astype(np.float64)
    var_back = (100 * F32(0.1) / 6) ** 2 + 0.3
    var_front = (100 * F32(0.12) / 5) ** 2 + 0.3
    a_front = _single_alpha(c, 64.0, 64.0, var_front, o[1]) * _tile_mask(c, 3, 4, 3, 4)
    r_back = math.ceil(3 * math.sqrt(var_back + math.sqrt(0.1)))
    t0, t1 = int((64 - r_back) // 16), int((64 + r_back) // 16)
    a_back = _single_alpha(c, 64.0, 64.0, var_back, o[0]) * _tile_mask(c, t0, t1, t0, t1)
    c_front = 0.5 + Y00 * dc[0].astype(np.float64)  # row 1 of the scene (z = 5) holds dc[0]
    c_back = 0.5 + Y00 * dc[1].astype(np.float64)
    expect = a_front[:, None] * c_front + ((1 - a_front) * a_back)[:, None] * c_back
    np.testing.assert_allclose(r["rgb"], expect, atol=1e-12)
    np.testing.assert_allclose(r["depth"], 5 * a_front + 6 * (1 - a_front) * a_back, atol=1e-12)
    np.testing.assert_allclose(r["final_T"], (1 - a_front) * (1 - a_back), atol=1e-12)
    # blended count: one per Gaussian whose alpha reaches the floor at the pixel
    np.testing.assert_array_equal(r["n_blend"], (a_front >= 1 / 255).astype(int) + (a_back >= 1 / 255).astype(int))


def test_separated_gaussians_are_independent(oracle):
    sc2 = scene_of([[-1.5, -1.5, 5], [1.5, 1.5, 5]], [[0.1] * 3] * 2, opacities=[0.8, 0.9],
                   dc=[[0.1, 0.2, 0.3], [0.3, 0.2, 0.1]])
    c = cam()
    both = oracle.render(sc2, c, np.eye(4), geom64=True)
    a = oracle.render(scene_of(sc2["means"][:1], sc2["scales"][:1], opacities=[0.8], dc=[[0.1, 0.2, 0.3]]),
                      c, np.eye(4), geom64=True)
    b = oracle.render(scene_of(sc2["means"][1:], sc2["scales"][1:], opacities=[0.9], dc=[[0.3, 0.2, 0.1]]),
                      c, np.eye(4), geom64=True)
    np.testing.assert_allclose(both["rgb"], a["rgb"] + b["rgb"], atol=1e-14)


def test_alpha_floor_boundary(oracle):
    # centre on a pixel centre (u = v = 64.5): alpha there equals the opacity
    z, f = 5.0, 100.0
    m = [[0.5 * z / f, 0.5 * z / f, z]]
    c = cam()
    below = oracle.render(scene_of(m, [[0.1] * 3], opacities=[(1 / 255) * (1 - 1e-6)], dc=[[0, 0, 0]]),
                          c, np.eye(4), geom64=True)
    above = oracle.render(scene_of(m, [[0.1] * 3], opacities=[(1 / 255) * (1 + 1e-6)], dc=[[0, 0, 0]]),
                          c, np.eye(4), geom64=True)
    assert below["alpha"].max() == 0.0
    assert (above["alpha"] > 0).sum() == 1
    assert above["alpha"][64 * 128 + 64] == pytest.approx(1 / 255, rel=2e-6)


def test_alpha_cap_and_transmittance_cutoff(oracle):
    # three capped Gaussians (alpha = 0.99) on one pixel centre: the third would take T
    # below 1e-4 and is not blended; last_idx = 2, final T = (1 - 0.99)^2
    z = np.array([5.0, 6.0, 7.0])
    m = np.stack([0.5 * z / 100, 0.5 * z / 100, z], 1)
    dc = np.array([[0.2, 0, 0], [0, 0.2, 0], [0, 0, 0.2]], np.float32)
    sc = scene_of(m, [[0.1] * 3] * 3, opacities=[0.999] * 3, dc=dc)
    r = oracle.render(sc, cam(), np.eye(4), geom64=True)
    p = 64 * 128 + 64
    c1, c2 = 0.5 + Y00 * dc[0].astype(np.float64), 0.5 + Y00 * dc[1].astype(np.float64)
    np.testing.assert_allclose(r["rgb"][p], 0.99 * c1 + (1 - 0.99) * 0.99 * c2, rtol=1e-14)
    assert r["last_idx"][p] == 2 and r["n_eval"][p] == 3 and r["n_blend"][p] == 2
    assert r["final_T"][p] == pytest.approx((1 - 0.99) ** 2, rel=1e-12)
    assert r["flags"][p] & oracle.TIE_T_CUTOFF  # T after two is within rounding of the cutoff


def _with_feats(sc, feats):
    sc = dict(sc)
    sc["feats_bf16"] = synth.to_bf16_bits(np.asarray(feats, np.float32))
    return sc


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_weights_telescope(oracle, seed):
    # feature == 1 makes F = sum of blending weights; F + T_final = 1 (telescoping product)
    sc = synth.tiny_scene(seed, sh_degree=1)
    sc = _with_feats(sc, np.ones((sc["means"].shape[0], 2)))
    r = oracle.render(sc, synth.tiny_camera(), np.eye(4), geom64=True)
    np.testing.assert_allclose(r["feats"][:, 0] + r["final_T"], 1.0, atol=1e-12)
    assert r["final_T"].min() >= 1e-4 and r["final_T"].max() <= 1.0
    assert r["alpha"].min() >= 0.0 and r["alpha"].max() < 1.0
    assert np.all(r["last_idx"] <= r["n_eval"])
    # blended Gaussians: never more than the examined prefix, none exactly when nothing was blended
    assert np.all(r["n_blend"] <= r["last_idx"])
    np.testing.assert_array_equal(r["n_blend"] == 0, r["last_idx"] == 0)


def test_features_identical_blending(oracle):
    # features equal to the colours (exact in bfloat16) reproduce the colour image
    g = np.random.default_rng(3)
    sc = synth.tiny_scene(4)
    n = sc["means"].shape[0]
    rgb = g.choice([0.25, 0.5, 0.75, 1.0], size=(n, 3)).astype(np.float32)
    sc["sh"][:, 0, :] = (rgb - 0.5) / np.float32(Y00)
    sc = _with_feats(sc, np.concatenate([rgb, np.zeros((n, 1), np.float32)], 1))
    r = oracle.render(sc, synth.tiny_camera(), np.eye(4), geom64=True)
    np.testing.assert_allclose(r["feats"][:, :3], r["rgb"], atol=1e-6)
    np.testing.assert_allclose(r["feats"][:, 3], 0.0, atol=0)


def test_unrounded_features_are_blended_like_the_bf16_ones(oracle):
    # the binary32 feature input (used to separate the error of bf16 storage):
    # given the bf16 values it reproduces the bf16 render exactly, and by
    # linearity in the features the storage error is the render of the
    # rounding residuals
    g = np.random.default_rng(11)
    sc = synth.tiny_scene(6, sh_degree=1)
    n = sc["means"].shape[0]
    f = g.standard_normal((n, 8)).astype(np.float32)
    sc = _with_feats(sc, f)
    fb = synth.bf16_bits_to_f32(sc["feats_bf16"])
    cam = synth.tiny_camera()
    rb = oracle.render(sc, cam, np.eye(4), geom64=True)
    same = dict(sc, feats_f32=fb)
    r1 = oracle.render(oracle.OracleScene(same, unrounded_feats=True), cam, np.eye(4), geom64=True)
    np.testing.assert_array_equal(r1["feats"], rb["feats"])
    np.testing.assert_array_equal(r1["rgb"], rb["rgb"])
    r32 = oracle.render(oracle.OracleScene(dict(sc, feats_f32=f), unrounded_feats=True), cam, np.eye(4),
                        geom64=True)
    resid = oracle.render(oracle.OracleScene(dict(sc, feats_f32=(f - fb).astype(np.float32)),
                                             unrounded_feats=True), cam, np.eye(4), geom64=True)
    np.testing.assert_allclose(r32["feats"] - rb["feats"], resid["feats"], rtol=0, atol=1e-15)
    assert np.abs(resid["feats"]).max() > 0


def test_depth_of_flat_scene(oracle):
    sc = synth.tiny_scene(5)
    sc["means"][:, 2] = 6.0
    r = oracle.render(sc, synth.tiny_camera(), np.eye(4), geom64=True)
    np.testing.assert_allclose(r["depth"], 6.0 * r["alpha"], atol=1e-12)


@pytest.mark.parametrize("seed,w,h,deg", [(0, 128, 128, 0), (1, 100, 75, 3), (2, 37, 129, 2)])
def test_binned_equals_brute_force(oracle, seed, w, h, deg):
    sc = synth.tiny_scene(seed, n=600, sh_degree=deg)
    c = cam(w, h, 110.0, w / 2 + 0.3, h / 2 - 0.7)
    for geom64 in (False, True):
        a = oracle.render(sc, c, np.eye(4), geom64=geom64)
        b = oracle.render(sc, c, np.eye(4), geom64=geom64, brute=True)
        for k in ("rgb", "depth", "final_T", "last_idx", "n_eval", "n_blend"):
            np.testing.assert_array_equal(a[k], b[k])


def test_pixel_subset_and_threads_agree(oracle):
    sc = synth.tiny_scene(6, sh_degree=3)
    c = synth.tiny_camera()
    full = oracle.render(sc, c, np.eye(4), n_threads=1)
    pix = np.random.default_rng(0).choice(128 * 128, 999, replace=False)
    sub = oracle.render(sc, c, np.eye(4), n_threads=4, pixels=pix)
    np.testing.assert_array_equal(sub["rgb"], full["rgb"][pix])
    np.testing.assert_array_equal(sub["last_idx"], full["last_idx"][pix])


def test_geom32_close_to_geom64(oracle):
    sc = synth.tiny_scene(8, sh_degree=3)
    c = synth.tiny_camera()
    a = oracle.render(sc, c, np.eye(4), geom64=False)
    b = oracle.render(sc, c, np.eye(4), geom64=True)
    ok = (a["flags"] | b["flags"]) & oracle.TIE_IMAGE == 0
    assert ok.mean() > 0.99
    np.testing.assert_allclose(a["rgb"][ok], b["rgb"][ok], atol=1e-4)


def test_empty_scene_and_all_culled(oracle):
    c = cam(40, 24)
    e = oracle.render(scene_of(np.zeros((0, 3)), np.zeros((0, 3))), c, np.eye(4))
    assert np.all(e["final_T"] == 1.0) and np.all(e["rgb"] == 0.0) and e["n_pairs"] == 0
    behind = oracle.render(scene_of([[0, 0, -5], [0, 0, 0.1]], [[0.1] * 3] * 2), c, np.eye(4))
    assert np.all(behind["final_T"] == 1.0) and behind["n_pairs"] == 0
