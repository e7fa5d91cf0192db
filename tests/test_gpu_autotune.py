"""Launch configurations and the autotuner (the coarse-to-fine pyramid of
Sec. 3.4 renders views of very different sizes), through the C ABI.

Every compositor variant, persistent grid and projection-side grid must give
the same bits as the defaults: the blending order and every reduction order
are fixed by the tile lists. The tuner's choice must not be slower than the
defaults it timed, must be what the scene then uses, and must survive a save
and a load of the cache file.
"""
import math

import numpy as np
import pytest
import torch

from paper_2507_15683_gb300 import synth

pytestmark = pytest.mark.gpu


def _scene(feat_dim=32):
    return synth.aerial_scene(81, 30000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20, feat_dim=feat_dim)


def _views():
    cams = [synth.camera(240, 136, 175.0), synth.camera(120, 68, 87.5), synth.camera(120, 68, 87.5)]
    poses = [synth.look_pose((100.0 + 10 * k, 40.0, 60.0), 0.3 * k, math.radians(30.0)) for k in range(3)]
    return cams, poses


def _render_all(gsr, S, cams, poses, feats):
    outs = [S.alloc_outputs(c, feat_dim=32 if feats else 0) for c in cams]
    S.render_batch(cams, poses, outs)
    single = S.render(cams[0], poses[0], S.alloc_outputs(cams[0], feat_dim=32 if feats else 0))
    torch.cuda.synchronize()
    return [{k: v.clone() for k, v in o.items()} for o in outs] + [{k: v.clone() for k, v in single.items()}]


def _grad_all(gsr, S, cams, poses, targets):
    qs = [synth.perturb_pose(T, synth.rng(90 + k), 0.5, 0.5) for k, T in enumerate(poses)]
    loss, grad = S.render_pose_grad_batch(cams, qs, [a for a, _ in targets], [b for _, b in targets])
    l1, g1 = S.render_pose_grad(cams[0], qs[0], targets[0][0], targets[0][1])
    return np.concatenate([np.asarray(loss, np.float64).ravel(), np.asarray(grad, np.float64).ravel(), [l1],
                           np.asarray(g1, np.float64)])


def _same(a, b):
    for x, y in zip(a, b):
        for k in x:
            torch.testing.assert_close(x[k], y[k], rtol=0, atol=0, msg=k)


def test_every_configuration_gives_the_default_bits(gsr):
    S = gsr.Scene(_scene())
    cams, poses = _views()
    shapes = [cams, cams[:1]]  # the batch and the single view: two call shapes
    ref = _render_all(gsr, S, cams, poses, True)
    ref_nf = _render_all(gsr, S, cams, poses, False)
    targets = [(o["rgb"], o["depth"]) for o in ref_nf[:3]]
    ref_g = _grad_all(gsr, S, cams, poses, targets)
    for mode, feats in ((gsr.GS_MODE_FORWARD, False), (gsr.GS_MODE_FEATURES, True), (gsr.GS_MODE_POSE_GRAD, None)):
        for v in range(gsr.GS_COMPOSITE_VARIANTS):
            occ = gsr.gs_scene_get_launch(S.handle, mode, cams)
            for per_sm, gm in ((0, 8), (1, 2), (2, 32)):
                for sh in shapes:
                    gsr.gs_scene_set_launch(S.handle, mode, sh, v, per_sm, gm)
                got = gsr.gs_scene_get_launch(S.handle, mode, cams)
                assert got["variant"] == v and got["grid_mult"] == gm and got["batch"] > 0
                assert got["ctas_per_sm"] == (per_sm if 0 < per_sm < got["occupancy"] else got["occupancy"])
                if feats is None:
                    np.testing.assert_array_equal(_grad_all(gsr, S, cams, poses, targets), ref_g)
                else:
                    _same(_render_all(gsr, S, cams, poses, feats), ref if feats else ref_nf)
        for sh in shapes:
            gsr.gs_scene_set_launch(S.handle, mode, sh, 0, 0, 8)
    S.close()


def test_autotune_picks_a_configuration_and_keeps_the_bits(gsr, tmp_path):
    S = gsr.Scene(_scene())
    cams, poses = _views()
    ref = _render_all(gsr, S, cams, poses, True)
    results = {}
    for mode in (gsr.GS_MODE_FORWARD, gsr.GS_MODE_FEATURES, gsr.GS_MODE_POSE_GRAD):
        r = gsr.gs_autotune(S.handle, mode, cams, poses, reps=3)
        print("mode", mode, r)
        assert r["candidates"] >= 8 and 0 < r["ms_best"] <= r["ms_default"]
        assert gsr.gs_scene_get_launch(S.handle, mode, cams) == r["best"]
        results[mode] = r["best"]
    _same(_render_all(gsr, S, cams, poses, True), ref)
    # the cache file: another scene on this device picks the same configurations up
    path = str(tmp_path / "launch.txt")
    gsr.gs_tune_save(S.handle, path)
    S2 = gsr.Scene(_scene())
    assert gsr.gs_tune_load(S2.handle, path) == 3
    for mode, best in results.items():
        assert gsr.gs_scene_get_launch(S2.handle, mode, cams) == best
    # lines of other devices are kept and ignored
    with open(path, "a") as f:
        f.write("Some Other GPU/8|2|%s|3 1 4\n" % "120x68*2,240x136*1")
    gsr.gs_tune_save(S2.handle, path)
    assert "Some Other GPU/8" in open(path).read()
    assert gsr.gs_tune_load(S2.handle, path) == 3
    S.close()
    S2.close()


def test_launch_arguments(gsr):
    S = gsr.Scene(_scene(0))
    cams, _ = _views()
    for bad in ((5, 0, 8), (0, -1, 8), (0, 0, 0), (0, 0, 65)):
        with pytest.raises(gsr.GsError) as e:
            gsr.gs_scene_set_launch(S.handle, gsr.GS_MODE_FORWARD, cams, *bad)
        assert e.value.status == gsr.GS_ERR_INVALID_ARG
    with pytest.raises(gsr.GsError) as e:
        gsr.gs_scene_get_launch(S.handle, 7, cams)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    with pytest.raises(gsr.GsError) as e:  # a scene without features has no feature mode to tune
        gsr.gs_autotune(S.handle, gsr.GS_MODE_FEATURES, cams[:1], [np.eye(4)])
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    with pytest.raises(gsr.GsError) as e:
        gsr.gs_tune_load(S.handle, "/nonexistent/launch.txt")
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    S.close()
