"""Pins of the oracle's loss, pose gradient and pose utilities.

The loss is the project's reading of the refinement objective: mean L1 over
the three colour channels plus 0.1 x mean L1 of the rendered depth, with the
gradient taken with respect to a left se(3) perturbation xi = (rho, phi) of
the world-to-camera pose. The oracle's forward-mode gradient is pinned against
central finite differences of its own binary64 loss, taken only where every
discrete decision (tile lists and order, skipped/blended/stopped Gaussians,
clamps, residual signs) is identical at +h and -h. Algorithm 2 of the paper
fixes the pose-difference angle.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from paper_2507_15683_gb300 import synth
from tests.oracle_scenes import rot_z


def _small_aerial(seed):
    sc = synth.aerial_scene(seed, 30000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20)
    cam = synth.camera(240, 136, 175.0)
    T_gt = synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0))
    return sc, cam, T_gt


def _workloads():
    out = []
    sc = synth.tiny_scene(11, n=500, sh_degree=3)
    sc["sh"][:, 1:, :] *= 4.0  # make view dependence matter
    out.append(("tiny", sc, synth.tiny_camera(), np.eye(4)))
    sc, cam, T = _small_aerial(12)
    out.append(("aerial", sc, cam, T))
    return out


def _fd_gradient(O, sc, cam, T, trgb, tdep, pw=None):
    base = O.render(sc, cam, T, geom64=True, want_grad=True, target_rgb=trgb, target_depth=tdep,
                    pixel_weight=pw, n_threads=4)
    fd = np.zeros(6)
    for k in range(6):
        for h in (1e-6, 1e-7, 1e-8, 1e-9):
            xi = np.zeros(6)
            xi[k] = h
            rp = O.render(sc, cam, O.se3_exp_left(xi, T), geom64=True, target_rgb=trgb, target_depth=tdep,
                          pixel_weight=pw, n_threads=4)
            rm = O.render(sc, cam, O.se3_exp_left(-xi, T), geom64=True, target_rgb=trgb, target_depth=tdep,
                          pixel_weight=pw, n_threads=4)
            if rp["signature"] == rm["signature"] == base["signature"]:
                fd[k] = (rp["loss"] - rm["loss"]) / (2 * h)
                break
        else:
            pytest.fail("no step keeps every discrete decision fixed for component %d" % k)
    return base, fd


@pytest.mark.parametrize("name,sc,cam,T_gt", _workloads(), ids=lambda x: x if isinstance(x, str) else "")
def test_forward_mode_gradient_matches_finite_differences(oracle, name, sc, cam, T_gt):
    tgt = oracle.render(sc, cam, T_gt, geom64=True)
    H, W = cam["height"], cam["width"]
    trgb = tgt["rgb"].T.reshape(3, H, W).astype(np.float32)
    tdep = tgt["depth"].reshape(H, W).astype(np.float32)
    T_q = synth.perturb_pose(T_gt, np.random.default_rng(3), 0.5, 0.05 if name == "tiny" else 0.5)
    pw = np.random.default_rng(4).uniform(0.0, 1.0, (H, W)).astype(np.float32)
    for weight in (None, pw):
        base, fd = _fd_gradient(oracle, sc, cam, T_q, trgb, tdep, weight)
        g = base["grad"]
        assert np.abs(g).max() > 1e-6
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_loss_is_zero_at_reference_pose_and_descends(oracle):
    sc, cam, T_gt = _small_aerial(13)
    tgt = oracle.render(sc, cam, T_gt, geom64=True)
    H, W = cam["height"], cam["width"]
    trgb = tgt["rgb"].T.reshape(3, H, W).astype(np.float32)
    tdep = tgt["depth"].reshape(H, W).astype(np.float32)
    at_gt = oracle.render(sc, cam, T_gt, geom64=True, target_rgb=trgb, target_depth=tdep)
    assert at_gt["loss"] < 1e-6
    T_q = synth.perturb_pose(T_gt, np.random.default_rng(5), 1.0, 1.0)
    r = oracle.render(sc, cam, T_q, geom64=True, want_grad=True, target_rgb=trgb, target_depth=tdep, n_threads=4)
    g = r["grad"]
    step = oracle.se3_exp_left(-1e-4 * g / np.linalg.norm(g), T_q)
    r2 = oracle.render(sc, cam, step, geom64=True, target_rgb=trgb, target_depth=tdep, n_threads=4)
    assert r2["loss"] < r["loss"]


def test_depth_weight_is_linear(oracle):
    sc, cam, T_gt = _small_aerial(14)
    tgt = oracle.render(sc, cam, T_gt, geom64=True)
    H, W = cam["height"], cam["width"]
    trgb = tgt["rgb"].T.reshape(3, H, W).astype(np.float32)
    tdep = tgt["depth"].reshape(H, W).astype(np.float32)
    T_q = synth.perturb_pose(T_gt, np.random.default_rng(6), 1.0, 1.0)
    res = [oracle.render(sc, cam, T_q, geom64=True, want_grad=True, target_rgb=trgb, target_depth=tdep,
                         depth_weight=w) for w in (0.0, 0.1, 0.2)]
    np.testing.assert_allclose(res[2]["grad"] - res[1]["grad"], res[1]["grad"] - res[0]["grad"], rtol=1e-9,
                               atol=1e-15)
    assert res[1]["loss"] - res[0]["loss"] == pytest.approx(res[2]["loss"] - res[1]["loss"], rel=1e-9)


def _twist(xi):
    rho, phi = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return M


def test_se3_exp_matches_matrix_exponential(oracle):
    g = np.random.default_rng(7)
    T0 = synth.aerial_pose()
    for scale in (1e-7, 1e-3, 0.5, 2.0):
        xi = g.standard_normal(6) * scale
        np.testing.assert_allclose(oracle.se3_exp_left(xi, T0), scipy.linalg.expm(_twist(xi)) @ T0,
                                   rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(oracle.se3_exp_left([0, 0, 0, 0, 0, math.pi / 2], np.eye(4)), rot_z(90), atol=1e-15)


def test_alg2_pose_difference(oracle):
    a, d = oracle.pose_diff(rot_z(90), np.eye(4))
    assert a == pytest.approx(90.0, abs=1e-12) and d == 0.0
    T = np.eye(4)
    T[:3, :3] = scipy.linalg.expm(_twist([0, 0, 0, math.radians(20), 0, 0]))[:3, :3]
    T[:3, 3] = [3, 4, 0]
    a, d = oracle.pose_diff(T, np.eye(4))
    assert a == pytest.approx(20.0, abs=1e-10) and d == pytest.approx(5.0)
    # trace slightly above 3 from rounding is clamped (no NaN)
    R = np.eye(4)
    R[0, 0] = 1 + 1e-12
    a, _ = oracle.pose_diff(R, np.eye(4))
    assert a == 0.0
