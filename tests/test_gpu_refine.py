"""Pose refinement driver (Adam on the se(3) tangent, left update) through the C ABI.

The pose-refinement workload: 500,000 aerial Gaussians at 960x540, query pose
2 deg / 5 m away from the reference; 50 iterations must bring the pose close
to the reference (angle by the paper's Algorithm 2 formula). The batched
driver must give exactly the poses of independent single-pose refinements.
"""
import math

import numpy as np
import pytest
import torch

from paper_2507_15683_gb300 import synth

pytestmark = pytest.mark.gpu


def _centre(T):
    T = np.asarray(T)
    return -T[:3, :3].T @ T[:3, 3]


def _targets(oracle, scene, cam, T):
    r = oracle.render(scene, cam, T, geom64=True, n_threads=16)
    H, W = cam["height"], cam["width"]
    return (torch.from_numpy(np.ascontiguousarray(r["rgb"].T.reshape(3, H, W), np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(r["depth"].reshape(H, W), np.float32)).cuda())


def test_refinement_converges_on_the_refine_workload(oracle, gsr):
    scene, cam, T_gt, T_q = synth.refine_workload()
    tr, td = _targets(oracle, scene, cam, T_gt)
    S = gsr.Scene(scene)
    p = gsr.pose(T_q)
    opts = gsr.gs_refine_defaults()
    hist = gsr.gs_refine_pose(S.handle, gsr.camera(cam), p, tr.data_ptr(), td.data_ptr(), None, opts,
                              torch.cuda.current_stream().cuda_stream)
    T_out = gsr.pose_matrix(p)
    a0, _ = oracle.pose_diff(T_q, T_gt)
    a1, _ = oracle.pose_diff(T_out, T_gt)
    d0 = np.linalg.norm(_centre(T_q) - _centre(T_gt))
    d1 = np.linalg.norm(_centre(T_out) - _centre(T_gt))
    print("angle %.3f -> %.3f deg, centre %.3f -> %.3f m, loss %.5f -> %.5f" % (a0, a1, d0, d1, hist[0], hist[-1]))
    assert hist[-1] < 0.5 * hist[0]
    assert a1 < 0.5 * a0 and d1 < 0.5 * d0
    S.close()


def test_batched_refinement_equals_single_refinements(oracle, gsr):
    scene = synth.aerial_scene(61, 30000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20)
    cams = [synth.camera(240, 136, 175.0), synth.camera(120, 68, 88.0), synth.camera(200, 100, 150.0)]
    refs = [synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0)),
            synth.look_pose((90.0, 60.0, 70.0), 0.7, math.radians(20.0)),
            synth.look_pose((110.0, 80.0, 65.0), 2.0, math.radians(35.0))]
    qs = [synth.perturb_pose(T, synth.rng(70 + k), 1.0, 1.0) for k, T in enumerate(refs)]
    tg = [_targets(oracle, scene, c, T) for c, T in zip(cams, refs)]
    S = gsr.Scene(scene)
    opts = gsr.gs_refine_defaults()
    opts.iterations = 8
    opts.lr_trans = 0.05
    stream = torch.cuda.current_stream().cuda_stream
    singles = []
    for c, T, (r, d) in zip(cams, qs, tg):
        p = gsr.pose(T)
        gsr.gs_refine_pose(S.handle, gsr.camera(c), p, r.data_ptr(), d.data_ptr(), None, opts, stream)
        singles.append(gsr.pose_matrix(p))
    poses = [gsr.pose(T) for T in qs]
    hist = gsr.gs_refine_poses_batch(S.handle, [gsr.camera(c) for c in cams], poses, [r.data_ptr() for r, _ in tg],
                                     [d.data_ptr() for _, d in tg], None, opts, stream)
    assert hist.shape == (3, 8)
    for k in range(3):
        np.testing.assert_array_equal(gsr.pose_matrix(poses[k]), singles[k])
    S.close()
