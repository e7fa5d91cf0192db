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


def _hat(xi):
    rho, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]]
    M[:3, 3] = rho
    return M


def test_device_adam_matches_a_host_adam_loop(oracle, gsr):
    """The device-side Adam step and Exp update against the same loop written
    here: gs_render_pose_grad for the gradient, Adam in numpy and the matrix
    exponential of the twist by scipy's expm."""
    expm = pytest.importorskip("scipy.linalg").expm
    scene = synth.aerial_scene(61, 30000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20)
    cam = synth.camera(240, 136, 175.0)
    ref = synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0))
    q = synth.perturb_pose(ref, synth.rng(71), 1.0, 1.0)
    r, d = _targets(oracle, scene, cam, ref)
    S = gsr.Scene(scene)
    opts = gsr.gs_refine_defaults()
    opts.iterations = 10
    opts.lr_trans = 0.05
    p = gsr.pose(q)
    hist = gsr.gs_refine_pose(S.handle, gsr.camera(cam), p, r.data_ptr(), d.data_ptr(), None, opts,
                              torch.cuda.current_stream().cuda_stream)
    T = np.array(q, np.float64)
    m = np.zeros(6)
    v = np.zeros(6)
    lr = np.array([opts.lr_trans] * 3 + [opts.lr_rot] * 3)
    losses = []
    for it in range(opts.iterations):
        loss, g = S.render_pose_grad(cam, T, r, d, depth_weight=opts.depth_weight)
        losses.append(loss)
        m = opts.beta1 * m + (1 - opts.beta1) * g
        v = opts.beta2 * v + (1 - opts.beta2) * g * g
        step = lr * (m / (1 - opts.beta1 ** (it + 1))) / (np.sqrt(v / (1 - opts.beta2 ** (it + 1))) + opts.eps)
        T = expm(_hat(-step)) @ T
    T_dev = gsr.pose_matrix(p)
    print("max |dR| %.3g, max |dt| %.3g m, loss rel %.3g" % (
        np.abs(T_dev[:3, :3] - T[:3, :3]).max(), np.abs(T_dev[:3, 3] - T[:3, 3]).max(),
        np.max(np.abs(np.array(hist) - losses) / np.array(losses))))
    # both loops take the same fp32 gradients while the poses agree to fp64
    # rounding; the tolerance covers a rounding-level pose difference carried
    # through a few fp32 gradients
    np.testing.assert_allclose(hist, losses, rtol=1e-6)
    np.testing.assert_allclose(T_dev[:3, :3], T[:3, :3], rtol=0, atol=1e-7)
    np.testing.assert_allclose(T_dev[:3, 3], T[:3, 3], rtol=0, atol=1e-5)
    S.close()


def test_device_refinement_restarts_when_a_later_pose_outgrows_the_workspace(gsr):
    """A nadir camera 5 m over a flat field of 100k Gaussians with a wide lens,
    a depth target of 1000 m everywhere and a translation rate of 500 m: the
    first Adam step lifts the camera to about 505 m, where it sees the whole
    field. The first pass needs a few thousand records, the later ones more
    than the scene's first workspace (65,536 records), so the device loop
    overflows in a replayed iteration, doubles the workspace, restarts from the
    caller's pose, and must still agree with the loop written here."""
    n = 100_000
    scene = synth.aerial_scene(62, n, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=1, building_frac=0.0)
    scene["means"][:, 2] = synth.rng(63).normal(0.0, 0.2, n).astype(np.float32)
    cam = synth.camera(240, 136, 40.0)
    q = synth.look_pose((100.0, 100.0, 5.0), 0.0, 0.0)
    S = gsr.Scene(scene)
    H = gsr.Scene(scene)
    out = S.render(cam, q)
    r = out["rgb"].clone()
    d = torch.full_like(out["depth"], 1000.0)
    opts = gsr.gs_refine_defaults()
    opts.iterations = 3
    opts.lr_trans = 500.0
    opts.lr_rot = 0.0
    opts.depth_weight = 10.0
    T = np.array(q, np.float64)
    m = np.zeros(6)
    v = np.zeros(6)
    lr = np.array([opts.lr_trans] * 3 + [opts.lr_rot] * 3)
    losses, needs = [], []
    for it in range(opts.iterations):
        loss, g = H.render_pose_grad(cam, T, r, d, depth_weight=opts.depth_weight)
        needs.append(H.status()[1])
        losses.append(loss)
        m = opts.beta1 * m + (1 - opts.beta1) * g
        v = opts.beta2 * v + (1 - opts.beta2) * g * g
        step = lr * (m / (1 - opts.beta1 ** (it + 1))) / (np.sqrt(v / (1 - opts.beta2 ** (it + 1))) + opts.eps)
        w = -step[3:]
        assert not w.any()
        T = T.copy()
        T[:3, 3] -= step[:3]  # Exp of a pure translation twist
    print("records needed per pass", needs, "camera height %.1f m" % (-(T[:3, :3].T @ T[:3, 3]))[2])
    assert needs[0] < 65536 < max(needs[1:])
    p = gsr.pose(q)
    hist = gsr.gs_refine_pose(S.handle, gsr.camera(cam), p, r.data_ptr(), d.data_ptr(), None, opts,
                              torch.cuda.current_stream().cuda_stream)
    np.testing.assert_allclose(hist, losses, rtol=1e-6)
    np.testing.assert_allclose(gsr.pose_matrix(p), T, rtol=0, atol=1e-6)
    # the same through the batched driver, beside a second view that stays small
    q2 = synth.look_pose((50.0, 50.0, 8.0), 0.3, 0.0)
    o2 = S.render(cam, q2)
    p_single = gsr.pose(q2)
    gsr.gs_refine_pose(S.handle, gsr.camera(cam), p_single, o2["rgb"].data_ptr(), o2["depth"].data_ptr(), None,
                       opts, torch.cuda.current_stream().cuda_stream)
    poses = [gsr.pose(q), gsr.pose(q2)]
    hb = gsr.gs_refine_poses_batch(S.handle, [gsr.camera(cam)] * 2, poses, [r.data_ptr(), o2["rgb"].data_ptr()],
                                   [d.data_ptr(), o2["depth"].data_ptr()], None, opts,
                                   torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(gsr.pose_matrix(poses[0]), gsr.pose_matrix(p))
    np.testing.assert_array_equal(gsr.pose_matrix(poses[1]), gsr.pose_matrix(p_single))
    np.testing.assert_array_equal(hb[0], hist)
    S.close()
    H.close()
