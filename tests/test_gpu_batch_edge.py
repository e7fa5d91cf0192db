"""Batched rendering, graph replay, edge cases and error handling through the C ABI."""
import math

import numpy as np
import pytest
import torch

from paper_2507_15683_gb300 import synth
from tests.gpu_helpers import compare_images, to_numpy
from tests.oracle_scenes import scene_of

pytestmark = pytest.mark.gpu


def _views():
    cams = [synth.camera(120, 68, 90.0), synth.camera(240, 136, 175.0), synth.camera(97, 61, 70.0)]
    poses = [synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0)),
             synth.look_pose((80.0, 90.0, 80.0), 1.0, math.radians(10.0)),
             synth.look_pose((120.0, 60.0, 50.0), 2.5, math.radians(40.0))]
    return cams, poses


def _scene():
    return synth.aerial_scene(41, 30000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20)


def _eq(a, b):
    for k in a:
        torch.testing.assert_close(a[k], b[k], rtol=0, atol=0)


def test_batch_equals_single_views(gsr):
    scene = _scene()
    S = gsr.Scene(scene)
    cams, poses = _views()
    singles = [S.render(c, T) for c, T in zip(cams, poses)]
    outs = [S.alloc_outputs(c) for c in cams]
    S.render_batch(cams, poses, outs)
    for a, b in zip(outs, singles):
        _eq(a, b)
    S.close()


def test_graph_replay_follows_pose_updates(gsr):
    scene = _scene()
    S = gsr.Scene(scene)
    cams, poses = _views()
    S.reserve(200000, 2000000)
    outs = [S.alloc_outputs(c) for c in cams]
    S.render_batch(cams, poses, outs, graph=True)
    assert S.status()[0] == 0
    ref = [S.render(c, T) for c, T in zip(cams, poses)]
    for a, b in zip(outs, ref):
        _eq(a, b)
    poses2 = [synth.perturb_pose(T, synth.rng(k), 3.0, 2.0) for k, T in enumerate(poses)]
    S.render_batch(cams, poses2, outs, graph=True)  # replay with new poses
    assert S.status()[0] == 0
    ref2 = [S.render(c, T) for c, T in zip(cams, poses2)]
    for a, b in zip(outs, ref2):
        _eq(a, b)
    S.close()


def test_empty_scene_and_all_culled(gsr):
    cam = synth.camera(40, 24, 30.0)
    for sc in (scene_of(np.zeros((0, 3)), np.zeros((0, 3))), scene_of([[0, 0, -5], [0, 0, 0.1]], [[0.1] * 3] * 2)):
        S = gsr.Scene(sc)
        out = S.render(cam, np.eye(4))
        assert torch.all(out["final_T"] == 1) and torch.all(out["rgb"] == 0) and torch.all(out["last_idx"] == 0)
        S.close()


@pytest.mark.parametrize("w,h", [(1, 1), (17, 33), (16, 16), (300, 1)])
def test_ragged_and_degenerate_sizes(oracle, gsr, w, h):
    scene = synth.tiny_scene(3, n=500, sh_degree=1)
    cam = synth.camera(w, h, 60.0, w / 2 + 0.25, h / 2 - 0.25)
    S = gsr.Scene(scene)
    gpu = to_numpy(S.render(cam, np.eye(4)), h, w)
    orc = oracle.render(scene, cam, np.eye(4), geom64=True)
    compare_images(gpu, orc, oracle, min_ok=0.9)
    S.close()


def test_long_tile_list_uses_global_sort(oracle, gsr):
    # 6000 small Gaussians inside one tile's footprint: a list longer than the
    # shared-memory sort capacity
    g = synth.rng(4)
    n = 6000
    means = np.stack([g.uniform(-0.05, 0.05, n), g.uniform(-0.05, 0.05, n), g.uniform(4, 8, n)], 1)
    scene = scene_of(means, np.full((n, 3), 0.004), quats=g.standard_normal((n, 4)),
                     opacities=g.uniform(0.02, 0.2, n), dc=g.uniform(0, 1, (n, 3)))
    cam = synth.tiny_camera()
    S = gsr.Scene(scene)
    out = S.render(cam, np.eye(4))
    cov = oracle.cov3d_f32(scene["scales"], scene["quats"])
    ri, rf = oracle.project_f32(scene["means"], cov, cam, np.eye(4))
    ts, keys, gids = oracle.bin_tiles(ri, rf, cam)
    assert np.diff(ts).max() > 2048
    gts, gkeys, ggids = S.tile_lists(0, cam, len(keys) + 8)
    np.testing.assert_array_equal(gkeys, keys)
    np.testing.assert_array_equal(ggids, gids)
    compare_images(to_numpy(out, 128, 128), oracle.render(scene, cam, np.eye(4), geom64=True), oracle)
    S.close()


def test_large_gaussian_covers_every_tile(oracle, gsr):
    scene = scene_of([[0, 0, 5], [0.3, 0.1, 6]], [[3.0, 2.0, 0.5], [0.2, 0.2, 0.2]], opacities=[0.5, 0.9],
                     dc=[[0.2, 0.4, 0.6], [0.9, 0.1, 0.3]])
    cam = synth.camera(200, 150, 120.0)
    S = gsr.Scene(scene)
    gpu = to_numpy(S.render(cam, np.eye(4)), 150, 200)
    compare_images(gpu, oracle.render(scene, cam, np.eye(4), geom64=True), oracle)
    S.close()


def test_capacity_regrow_and_async_status(oracle, gsr):
    # 70,000 visible Gaussians exceed the first-call record guess (65,536)
    g = synth.rng(6)
    n = 70000
    means = np.stack([g.uniform(-2, 2, n), g.uniform(-2, 2, n), g.uniform(4, 8, n)], 1)
    scene = scene_of(means, np.full((n, 3), 0.03), opacities=np.full(n, 0.05), dc=g.uniform(0, 1, (n, 3)))
    cam = synth.tiny_camera()
    S = gsr.Scene(scene)
    out = S.render(cam, np.eye(4))  # synchronous: grows and re-renders
    compare_images(to_numpy(out, 128, 128), oracle.render(scene, cam, np.eye(4), geom64=True), oracle)
    S.close()
    S = gsr.Scene(scene)
    S.reserve(1000, 1000)
    S.render(cam, np.eye(4), sync=False)
    st, need_rec, _ = S.status()
    assert st == gsr.GS_ERR_CAPACITY and need_rec >= n
    S.close()


def test_invalid_arguments_return_errors(gsr):
    with pytest.raises(gsr.GsError) as e:
        bad = synth.tiny_scene(0)
        bad["sh_degree"] = 5
        gsr.Scene(bad)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    S = gsr.Scene(synth.tiny_scene(0))
    with pytest.raises(gsr.GsError) as e:
        S.render({"width": 0, "height": 4, "fx": 1, "fy": 1, "cx": 0, "cy": 0}, np.eye(4))
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    T = np.eye(4)
    T[0, 3] = float("nan")
    with pytest.raises(gsr.GsError) as e:
        S.render(synth.tiny_camera(), T)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    S.close()


def _targets_for(oracle, scene, cams, poses):
    out = []
    for c, T in zip(cams, poses):
        r = oracle.render(scene, c, T, geom64=True, n_threads=8)
        H, W = c["height"], c["width"]
        out.append((torch.from_numpy(np.ascontiguousarray(r["rgb"].T.reshape(3, H, W), np.float32)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(r["depth"].reshape(H, W), np.float32)).cuda()))
    return out


def test_batched_pose_gradient_equals_single_views(oracle, gsr):
    scene = _scene()
    cams, poses = _views()
    tg = _targets_for(oracle, scene, cams, poses)
    queries = [synth.perturb_pose(T, synth.rng(20 + k), 1.0, 1.0) for k, T in enumerate(poses)]
    weights = [None, torch.rand(cams[1]["height"], cams[1]["width"], device="cuda"), None]
    S = gsr.Scene(scene)
    single = [S.render_pose_grad(c, T, r, d, w, 0.1) for c, T, (r, d), w in zip(cams, queries, tg, weights)]
    loss, grad = S.render_pose_grad_batch(cams, queries, [r for r, _ in tg], [d for _, d in tg], weights, 0.1)
    for v, (l1, g1) in enumerate(single):
        assert loss[v] == l1
        np.testing.assert_array_equal(grad[v], g1)
    # graph replay with new poses writes the same numbers to the device buffer
    res = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    S.reserve(400000, 4000000)
    S.render_pose_grad_batch(cams, queries, [r for r, _ in tg], [d for _, d in tg], weights, 0.1, results=res,
                             graph=True)
    assert S.status()[0] == 0
    np.testing.assert_array_equal(res[:, 0].cpu().numpy(), loss)
    np.testing.assert_array_equal(res[:, 1:7].cpu().numpy(), grad)
    queries2 = [synth.perturb_pose(T, synth.rng(40 + k), 1.0, 1.0) for k, T in enumerate(poses)]
    S.render_pose_grad_batch(cams, queries2, [r for r, _ in tg], [d for _, d in tg], weights, 0.1, results=res,
                             graph=True)
    assert S.status()[0] == 0
    single2 = [S.render_pose_grad(c, T, r, d, w, 0.1) for c, T, (r, d), w in zip(cams, queries2, tg, weights)]
    for v, (l1, g1) in enumerate(single2):
        assert float(res[v, 0]) == l1
        np.testing.assert_array_equal(res[v, 1:7].cpu().numpy(), g1)
    S.close()


@pytest.mark.parametrize("n", [2, 20, 50, 100, 200, 256])
def test_short_lists_with_equal_depths(oracle, gsr, n):
    # n small Gaussians inside one 16 x 16 tile on three exact depth planes: the
    # warp sort must give ascending depth bits with ties in Gaussian-index order
    g = synth.rng(50 + n)
    z = g.choice([4.0, 5.0, 6.5], n)
    means = np.stack([g.uniform(-0.02, 0.02, n) * z, g.uniform(-0.02, 0.02, n) * z, z], 1)
    scene = scene_of(means, np.full((n, 3), 0.002), opacities=g.uniform(0.05, 0.3, n), dc=g.uniform(0, 1, (n, 3)))
    cam = synth.camera(64, 64, 300.0)
    S = gsr.Scene(scene)
    out = S.render(cam, np.eye(4))
    cov = oracle.cov3d_f32(scene["scales"], scene["quats"])
    ri, rf = oracle.project_f32(scene["means"], cov, cam, np.eye(4))
    ts, keys, gids = oracle.bin_tiles(ri, rf, cam)
    assert np.diff(ts).max() <= 256
    gts, gkeys, ggids = S.tile_lists(0, cam, len(keys) + 8)
    np.testing.assert_array_equal(gts, ts)
    np.testing.assert_array_equal(gkeys, keys)
    np.testing.assert_array_equal(ggids, gids)
    compare_images(to_numpy(out, 64, 64), oracle.render(scene, cam, np.eye(4), geom64=True), oracle)
    S.close()


def test_kernel_timing_changes_no_result(gsr):
    """With kernel timing on, the shading pass runs in order after the
    projection instead of beside the binning: images and the pose gradient
    must be bit-identical either way."""
    scene = _scene()
    cams, poses = _views()
    cam, T = cams[0], poses[0]
    S = gsr.Scene(scene)
    ref = S.render(cam, T)
    tr, td = ref["rgb"].clone(), ref["depth"].clone()
    Tq = synth.perturb_pose(T, synth.rng(5), 1.0, 1.0)
    a = S.render(cam, Tq)
    la, ga = S.render_pose_grad(cam, Tq, tr, td)
    gsr.gs_scene_set_timing(S.handle, True)
    b = S.render(cam, Tq)
    lb, gb = S.render_pose_grad(cam, Tq, tr, td)
    gsr.gs_scene_set_timing(S.handle, False)
    _eq(a, b)
    assert la == lb
    np.testing.assert_array_equal(ga, gb)
    S.close()
