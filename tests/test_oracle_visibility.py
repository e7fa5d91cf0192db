"""Pins of the oracle's render-gradient visibility check (Algorithm 1): the
binary64 mean gradient of the summed colours against finite differences and
against the camera-translation identity, and the structural cases (occluded,
outside the image); no GPU."""
import numpy as np
import pytest

from paper_2507_15683_gb300 import synth
from tests.oracle_scenes import scene_of


def _tiny():
    sc = synth.tiny_scene(11, n=400, sh_degree=1)
    sc["sh"][:, 1:, :] *= 3.0  # view-dependent colour: the colour rows of the gradient matter
    # a rotated, shifted camera, so that d p / d mean = R differs from the identity
    return sc, synth.tiny_camera(), synth.perturb_pose(np.eye(4), synth.rng(12), 3.0, 0.1)


def test_mean_gradient_matches_finite_differences(oracle):
    sc, cam, T = _tiny()
    base = oracle.render(sc, cam, T, geom64=True)
    # Gaussians that contribute somewhere: take a few of the largest footprints
    cov = oracle.cov3d_f32(sc["scales"], sc["quats"])
    ri, _ = oracle.project_f32(sc["means"], cov, cam, T)
    vis = np.nonzero(ri[:, oracle.I_STATUS] == oracle.VISIBLE)[0]
    area = (ri[vis, 2] - ri[vis, 1] + 1) * (ri[vis, 4] - ri[vis, 3] + 1)
    checked = 0
    for g in vis[np.argsort(-area)][:12]:
        r0 = oracle.mean_gradient(sc, cam, T, int(g))
        if not np.any(r0["grad"]):
            continue
        for a in range(3):
            vals, steps, sigs = [], [], []
            for sgn in (-1, 1):
                s2 = dict(sc)
                s2["means"] = sc["means"].copy()
                s2["means"][g, a] = np.float32(sc["means"][g, a] + sgn * 1e-4)
                steps.append(float(s2["means"][g, a]) - float(sc["means"][g, a]))
                r = oracle.mean_gradient(s2, cam, T, int(g))
                vals.append(r["sum"])
                sigs.append(r["signature"])
            if not (sigs[0] == sigs[1] == r0["signature"]):
                continue  # a discrete decision moved within +-h: no certified difference
            fd = (vals[1] - vals[0]) / (steps[1] - steps[0])
            assert fd == pytest.approx(r0["grad"][a], rel=2e-5, abs=1e-7 * max(1.0, abs(r0["sum"])))
            checked += 1
    assert checked >= 6
    assert base["rgb"].sum() > 0


def test_sum_of_mean_gradients_is_the_camera_translation_gradient(oracle):
    # moving every mean by d equals moving the camera by -d (camera-frame shift R d, view
    # directions shifted alike): sum_j grad_mean_j = R^T grad_rho of the summed colours
    sc, cam, T = _tiny()
    H, W = cam["height"], cam["width"]
    vis = oracle.visibility(sc, cam, T)
    total = vis["grad"].sum(axis=0)
    # grad_rho of sum C from the L1 loss with targets far above every colour (all signs -1)
    big = np.full((3, H, W), 1e6, np.float32)
    r = oracle.render(sc, cam, T, geom64=True, want_grad=True, target_rgb=big, target_depth=np.zeros((H, W),
                      np.float32), depth_weight=0.0)
    grad_rho = -3.0 * H * W * np.asarray(r["grad"][:3])
    np.testing.assert_allclose(total, np.asarray(T)[:3, :3].T @ grad_rho, rtol=1e-9, atol=1e-9)


def test_visibility_structural_cases(oracle):
    cam = synth.camera(128, 128, 100.0)
    # three wide walls (opacity 0.985) at z = 5, 5.5, 6 leave T < 1e-4 before a small
    # Gaussian at z = 8 on the axis can be reached anywhere in its tile: never blended.
    # A fifth Gaussian at z = 5 projects left of the image but its footprint reaches in.
    means = [[0, 0, 5.0], [0, 0, 5.5], [0, 0, 6.0], [0.01, 0.01, 8.0], [-3.3, 0.0, 5.0]]
    scales = [[10.0] * 3, [10.0] * 3, [10.0] * 3, [0.02] * 3, [0.3] * 3]
    sc = scene_of(means, scales, opacities=[0.985, 0.985, 0.985, 0.9, 0.9],
                  dc=[[0.5, 0.1, 0.1], [0.1, 0.5, 0.1], [0.1, 0.1, 0.5], [0.9, 0.9, 0.9], [0.2, 0.8, 0.2]])
    v = oracle.visibility(sc, cam, np.eye(4))
    assert v["M"][0] and v["M"][1]  # walls in front: visible
    assert not v["M_r"][3] and not np.any(v["grad"][3]) and v["M_i"][3] and not v["flag"][3]  # occluded
    assert v["M_r"][4] and not v["M_i"][4] and not v["M"][4]  # contributes, but projects outside
    assert v["uv"][4, 0] < 0
