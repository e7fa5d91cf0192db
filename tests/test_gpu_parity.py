"""GPU vs oracle parity of the forward path, through the C ABI.

Projection records and tile lists are compared bit for bit (binary32 discrete
layer); images element by element within 1e-4 of the fp64 oracle (relative to
each output's scale), on every pixel whose blending decisions are not within
rounding of a threshold; last-blended indices exactly on those pixels.
"""
import math

import numpy as np
import pytest

from paper_2507_15683_gb300 import synth
from tests.gpu_helpers import compare_images, to_numpy

pytestmark = pytest.mark.gpu


def _small_aerial(seed, n=30000, w=240, h=136, f=175.0):
    sc = synth.aerial_scene(seed, n, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20)
    cam = synth.camera(w, h, f)
    T = synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0))
    return sc, cam, T


CASES = {
    "tiny": lambda: (synth.tiny_scene(0), synth.tiny_camera(), np.eye(4)),
    "tiny_sh3_ragged": lambda: (synth.tiny_scene(1, n=2000, sh_degree=3), synth.camera(101, 77, 90.0, 50.3, 38.9),
                                np.eye(4)),
    "aerial_small": lambda: _small_aerial(21),
    "aerial_small_sh2": lambda: (dict(synth.aerial_scene(22, 20000, extent=(0, 200, 0, 200), n_clusters=10,
                                                         sh_degree=2)),
                                 synth.camera(250, 131, 180.0), synth.look_pose((90, 30, 70), 0.3, 0.6)),
}


def _check_records_and_lists(oracle, S, scene, cam, T):
    cov = oracle.cov3d_f32(scene["scales"], scene["quats"])
    ri, rf = oracle.project_f32(scene["means"], cov, cam, T)
    vis = np.nonzero(ri[:, oracle.I_STATUS] == oracle.VISIBLE)[0]
    rec = S.records(0, capacity=len(vis) + 1024)
    rec = rec[np.argsort(rec[:, 0])]
    np.testing.assert_array_equal(rec[:, 0], vis)
    np.testing.assert_array_equal(rec[:, 1:5], ri[vis, 1:5])
    np.testing.assert_array_equal(rec[:, 5].view(np.uint32), rf[vis, oracle.F_Z].view(np.uint32))
    # blending centre (float-float) against Algorithm 1 evaluated in binary64
    p = scene["means"][vis].astype(np.float64) @ np.asarray(T)[:3, :3].T + np.asarray(T)[:3, 3]
    k = {q: float(np.float32(cam[q])) for q in ("fx", "fy", "cx", "cy")}  # intrinsics are binary32 inputs
    u64 = k["fx"] * p[:, 0] / p[:, 2] + k["cx"]
    v64 = k["fy"] * p[:, 1] / p[:, 2] + k["cy"]
    f = rec[:, 6:10].view(np.float32).astype(np.float64)
    np.testing.assert_allclose(f[:, 0] + f[:, 1], u64, rtol=0, atol=1e-6)
    np.testing.assert_allclose(f[:, 2] + f[:, 3], v64, rtol=0, atol=1e-6)
    ts, keys, gids = oracle.bin_tiles(ri, rf, cam)
    gts, gkeys, ggids = S.tile_lists(0, cam, capacity=len(keys) + 16)
    np.testing.assert_array_equal(gts, ts)
    np.testing.assert_array_equal(gkeys, keys)
    np.testing.assert_array_equal(ggids, gids)
    return len(keys)


@pytest.mark.parametrize("case", sorted(CASES))
def test_forward_parity(oracle, gsr, case):
    scene, cam, T = CASES[case]()
    S = gsr.Scene(scene)
    out = S.render(cam, T)
    n_pairs = _check_records_and_lists(oracle, S, scene, cam, T)
    assert n_pairs > 0
    gpu = to_numpy(out, cam["height"], cam["width"])
    orc = oracle.render(scene, cam, T, geom64=True, n_threads=8)
    errs = compare_images(gpu, orc, oracle)
    # informational: against the oracle that blends with the binary32 centre/covariance
    orc32 = oracle.render(scene, cam, T, n_threads=8)
    ok = ((orc32["flags"] | orc["flags"]) & oracle.TIE_IMAGE) == 0
    print(case, "scaled errors vs fp64 oracle:", errs,
          "rgb vs binary32-geometry oracle: %.3g" % np.abs(gpu["rgb"] - orc32["rgb"])[ok].max())
    S.close()


def test_features_bf16_fp32_accumulation(oracle, gsr):
    scene, cam, T = _small_aerial(23, n=20000)
    g = synth.rng(5)
    f = g.standard_normal((scene["means"].shape[0], 32)).astype(np.float32)
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    scene["feats_bf16"] = synth.to_bf16_bits(f)
    S = gsr.Scene(scene)
    out = S.render(cam, T)
    gpu = to_numpy(out, cam["height"], cam["width"])
    orc = oracle.render(scene, cam, T, geom64=True, n_threads=8)
    errs = compare_images(gpu, orc, oracle)
    assert "feats" in errs
    # storage error of bf16, apart from the blending error gated above: the
    # oracle blending the unrounded binary32 vectors; reported, and bounded by
    # what rounding unit vectors (|f_i| < 1) to 8 significant bits can cost
    scene["feats_f32"] = f
    o32 = oracle.render(oracle.OracleScene(scene, unrounded_feats=True), cam, T, geom64=True, n_threads=8)
    ok = (orc["flags"] & oracle.TIE_IMAGE) == 0
    store = np.abs(orc["feats"][ok] - o32["feats"][ok])
    blend = np.abs(gpu["feats"][ok] - orc["feats"][ok])
    print("features: bf16 storage max %.3g rms %.3g; fp32 blending max %.3g rms %.3g"
          % (store.max(), np.sqrt((store ** 2).mean()), blend.max(), np.sqrt((blend ** 2).mean())))
    assert 0 < store.max() <= 2.0 ** -9 and blend.max() < store.max()
    S.close()


def test_full_size_aerial_1080p(oracle, gsr):
    """1,000,000 Gaussians at 1920x1080 in the benchmark's launch configuration:
    records and tile lists bit for bit, images on 20,000 sampled pixels."""
    scene = synth.aerial_scene(2, 1_000_000)
    cam = synth.aerial_camera()
    T = synth.aerial_pose()
    S = gsr.Scene(scene)
    out = S.render(cam, T)
    n_pairs = _check_records_and_lists(oracle, S, scene, cam, T)
    assert n_pairs > 500_000
    gpu = to_numpy(out, cam["height"], cam["width"])
    pix = np.sort(synth.rng(9).choice(cam["width"] * cam["height"], 20000, replace=False))
    orc = oracle.render(scene, cam, T, pixels=pix, geom64=True, n_threads=16)
    compare_images(gpu, orc, oracle, pixels=pix)
    S.close()


def test_full_size_batched_84_views(oracle, gsr):
    """The 84-view mixed-resolution batch (2,000,000 Gaussians in 4 partitions,
    32 BF16 feature channels) in the graph launch the benchmark times: one view
    of each resolution against the oracle on sampled pixels, features included,
    and every view bit-identical to its single-view render."""
    import torch
    scene = synth.partitioned_scene(4, 2, 2, 500_000, sh_degree=3, feat_dim=32)
    cams, poses = synth.batched_views()
    S = gsr.Scene(scene)
    outs = [S.alloc_outputs(c, feat_dim=32) for c in cams]
    S.render_batch(cams, poses, outs)  # sizes the workspace
    _, n_rec, n_pairs = S.status()
    S.reserve(int(n_rec * 1.2) + 1024, int(n_pairs * 1.2) + 4096)
    S.render_batch(cams, poses, outs, graph=True)
    assert S.status()[0] == 0
    for v in (0, 64, 80):  # 480x270, 960x540, 1920x1080
        cam, T = cams[v], poses[v]
        H, W = cam["height"], cam["width"]
        gpu = to_numpy(outs[v], H, W)
        pix = np.sort(synth.rng(90 + v).choice(W * H, min(W * H, 6000), replace=False))
        orc = oracle.render(scene, cam, T, pixels=pix, geom64=True, n_threads=16)
        errs = compare_images(gpu, orc, oracle, pixels=pix)
        assert "feats" in errs
        single = S.alloc_outputs(cam, feat_dim=32)
        S.render_batch([cam], [T], [single])
        for k in single:
            torch.testing.assert_close(single[k], outs[v][k], rtol=0, atol=0)
    S.close()


def test_full_size_pose_gradient_1080p(oracle, gsr):
    """The benchmark's pose-gradient step (1,000,000 Gaussians, 1920x1080, query
    2 deg / 5 m from the reference) on 20,000 sampled pixels: the loss and
    gradient restricted to those pixels (weight 1 there, 0 elsewhere) against the
    oracle's; near-tie pixels get weight 0 on both sides."""
    import torch
    from tests.gpu_helpers import GRAD_TOL, block_rel_err, component_rel_err
    scene = synth.aerial_scene(2, 1_000_000)
    cam = synth.aerial_camera()
    T_ref = synth.aerial_pose()
    T_q = synth.perturb_pose(T_ref, synth.rng(100), 2.0, 5.0)
    H, W = cam["height"], cam["width"]
    pix = np.sort(synth.rng(7).choice(W * H, 20000, replace=False))
    ref = oracle.render(scene, cam, T_ref, pixels=pix, geom64=True, n_threads=16)
    trgb = np.zeros((3, H * W), np.float32)
    tdep = np.zeros(H * W, np.float32)
    trgb[:, pix] = ref["rgb"].T
    tdep[pix] = ref["depth"]
    trgb, tdep = trgb.reshape(3, H, W), tdep.reshape(H, W)
    w = np.zeros(H * W, np.float32)
    w[pix] = 1.0
    probe = oracle.render(scene, cam, T_q, pixels=pix, geom64=True, target_rgb=trgb, target_depth=tdep,
                          pixel_weight=w.reshape(H, W), n_threads=16)
    w[pix] *= (probe["flags"] == 0)
    w = w.reshape(H, W)
    orc = oracle.render(scene, cam, T_q, pixels=pix, geom64=True, want_grad=True, target_rgb=trgb,
                        target_depth=tdep, pixel_weight=w, n_threads=16)
    S = gsr.Scene(scene)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss, grad = S.render_pose_grad(cam, T_q, t(trgb), t(tdep), t(w))
    S.close()
    assert loss == pytest.approx(orc["loss"], rel=1e-4)
    errs = block_rel_err(grad, orc["grad"])
    comp = component_rel_err(grad, orc["grad"])
    print("loss", loss, orc["loss"], "grad", grad, orc["grad"], "block rel err", errs, "component rel err", comp)
    assert max(errs) <= GRAD_TOL and max(comp) <= GRAD_TOL
