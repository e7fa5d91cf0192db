"""Partitioned and streamed scenes (Sec. 3.1 cells) through the C ABI.

Frustum culling of whole partitions must not change any result: tile lists
stay bit-identical to the oracle's (which projects every Gaussian) and images
stay within tolerance. A streamed scene uploads exactly the partitions its
views need, and renders like a device-resident one. The large-scene workload
(6M Gaussians, 16 partitions, SH degree 3 + 32 BF16 features, views from
480x270 to 3840x2160) is checked on sampled pixels, including the pose gradient.
"""
import math

import numpy as np
import pytest
import torch

from paper_2507_15683_gb300 import synth
from tests.gpu_helpers import GRAD_TOL, block_rel_err, compare_images, to_numpy

pytestmark = pytest.mark.gpu


N_PART = 16
PER_PART = 20_000


def _scene():
    # the large-scene layout (4 x 4 cells of 500 m) at a lower density
    return synth.partitioned_scene(7, 4, 4, PER_PART, cell_m=500.0, sh_degree=2, feat_dim=32)


def _views():
    cams = [synth.camera(240, 136, 175.0), synth.camera(160, 90, 120.0), synth.camera(200, 112, 150.0)]
    poses = [synth.look_pose((250.0, 250.0, 300.0), 0.0, 0.0),                      # nadir over a corner cell
             synth.look_pose((1700.0, 1700.0, 350.0), math.radians(225), math.radians(35.0)),
             synth.look_pose((1000.0, 1000.0, 400.0), 0.5, 0.0)]                    # nadir over the centre
    return cams, poses


def _keys(oracle, scene, cam, T):
    cov = oracle.cov3d_f32(scene["scales"], scene["quats"])
    ri, rf = oracle.project_f32(scene["means"], cov, cam, T)
    return oracle.bin_tiles(ri, rf, cam)


@pytest.mark.parametrize("streamed", [False, True])
def test_partition_culling_keeps_results(oracle, gsr, streamed):
    scene = _scene()
    cams, poses = _views()
    S = gsr.Scene(scene, stream_partitions=streamed)
    per_part = None
    for v, (c, T) in enumerate(zip(cams, poses)):
        out = S.render(c, T)
        ts, keys, gids = _keys(oracle, scene, c, T)
        gts, gkeys, ggids = S.tile_lists(0, c, len(keys) + 16)
        np.testing.assert_array_equal(gkeys, keys)
        np.testing.assert_array_equal(ggids, gids)
        compare_images(to_numpy(out, c["height"], c["width"]), oracle.render(scene, c, T, geom64=True, n_threads=16),
                       oracle)
        b, res, act = S.stream_stats()
        assert act < N_PART  # no view reaches every cell
        if streamed:
            per_part = PER_PART * (16 + 32 + 16 * 7 + 64)
            assert b == res * per_part
    S.close()


def test_streamed_scene_evict_and_batch(oracle, gsr):
    scene = _scene()
    cams, poses = _views()
    S = gsr.Scene(scene, stream_partitions=True)
    D = gsr.Scene(scene)
    outs = [S.alloc_outputs(c, feat_dim=32) for c in cams]
    S.render_batch(cams, poses, outs)
    b1, res1, act1 = S.stream_stats()
    assert res1 == act1  # the batch walked exactly the partitions it uploaded
    gsr.gs_scene_evict(S.handle)
    assert S.stream_stats()[1] == 0
    for c, T, o in zip(cams, poses, outs):
        ref = D.render(c, T)
        for k in ref:
            torch.testing.assert_close(o[k], ref[k], rtol=0, atol=0)
        again = S.render(c, T)
        for k in ref:
            torch.testing.assert_close(again[k], ref[k], rtol=0, atol=0)
    assert S.stream_stats()[0] > b1  # evicted partitions were uploaded again
    S.close()
    D.close()


def test_large_streamed_scene_pyramid(oracle, gsr):
    """6,000,000 Gaussians in 16 streamed partitions; one query pose at the two
    top pyramid levels (1920x1080, 3840x2160): tile lists bit for bit, images on
    sampled pixels, pose gradient on the same pixels vs the fp64 oracle."""
    scene = synth.partitioned_scene(5, 4, 4, 375_000, cell_m=500.0, sh_degree=3, feat_dim=32)
    S = gsr.Scene(scene, stream_partitions=True)
    T_ref = synth.look_pose((1000.0, 900.0, 300.0), 0.3, math.radians(25.0))
    T_q = synth.perturb_pose(T_ref, synth.rng(8), 1.0, 2.0)
    for level in (2, 3):
        f = 350.0 * 2 ** level
        cam = synth.camera(480 * 2 ** level, 270 * 2 ** level, f)
        H, W = cam["height"], cam["width"]
        out = S.render(cam, T_q)
        ts, keys, gids = _keys(oracle, scene, cam, T_q)
        gts, gkeys, ggids = S.tile_lists(0, cam, len(keys) + 16)
        np.testing.assert_array_equal(gkeys, keys)
        np.testing.assert_array_equal(ggids, gids)
        pix = np.sort(synth.rng(level).choice(H * W, 3000, replace=False))
        orc = oracle.render(scene, cam, T_q, pixels=pix, geom64=True, n_threads=16)
        errs = compare_images(to_numpy(out, H, W), orc, oracle, pixels=pix)
        print("level", level, "pairs", len(keys), "errors", errs, "stream", S.stream_stats())
        # pose gradient on the sampled pixels (weight 1 there, 0 elsewhere and at near ties)
        tgt = oracle.render(scene, cam, T_ref, pixels=pix, geom64=True, n_threads=16)
        trgb = np.zeros((3, H * W), np.float32)
        tdep = np.zeros(H * W, np.float32)
        trgb[:, pix] = tgt["rgb"].T
        tdep[pix] = tgt["depth"]
        w = np.zeros(H * W, np.float32)
        w[pix] = 1.0
        probe = oracle.render(scene, cam, T_q, pixels=pix, geom64=True, target_rgb=trgb.reshape(3, H, W),
                              target_depth=tdep.reshape(H, W), pixel_weight=w.reshape(H, W), n_threads=16)
        w[pix] = (probe["flags"] == 0).astype(np.float32)
        ref = oracle.render(scene, cam, T_q, pixels=pix, geom64=True, want_grad=True,
                            target_rgb=trgb.reshape(3, H, W), target_depth=tdep.reshape(H, W),
                            pixel_weight=w.reshape(H, W), n_threads=16)
        t = lambda a, *sh: torch.from_numpy(np.ascontiguousarray(a).reshape(*sh)).cuda()
        loss, grad = S.render_pose_grad(cam, T_q, t(trgb, 3, H, W), t(tdep, H, W), t(w, H, W))
        assert loss == pytest.approx(ref["loss"], rel=1e-4)
        e = block_rel_err(grad, ref["grad"])
        print("level", level, "grad block rel err", e)
        assert max(e) <= GRAD_TOL
    S.close()
