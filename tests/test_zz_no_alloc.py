"""gs_render_noalloc: the forward render that takes all of its working memory
from the library's fixed device array instead of allocating it.

It is for callers that may not allocate device memory when they render (a
pre-sized service, a plug-in whose host owns device memory, code running
beside a global-mode graph capture). It runs the same kernels on the same
inputs as gs_render, so its outputs must equal gs_render's bit for bit, on
calls in a row: the shared array keeps the previous call's contents, so a
smaller view after a larger one, and the larger one again after the smaller,
check in both orders that everything that must start at zero is cleared.
This file is collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest
import torch

from paper_2507_15683_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_desc(gsr, scene, keep):
    def t(x, dtype):
        a = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()
        keep.append(a)
        return a.data_ptr()

    n = scene["means"].shape[0]
    f = scene.get("feats_bf16")
    fp = 0 if f is None else t(np.asarray(f).view(np.int16), torch.int16)
    return gsr.gs_scene_desc(n, scene["sh_degree"], 0 if f is None else 32, t(scene["means"], torch.float32),
                             t(scene["scales"], torch.float32), t(scene["quats"], torch.float32),
                             t(scene["opacities"], torch.float32), t(scene["sh"], torch.float32), fp, 0, None, 1)


def _scene():
    scene = synth.aerial_scene(51, 20000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=10)
    f = synth.rng(52).standard_normal((20000, 32)).astype(np.float32)
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    scene["feats_bf16"] = synth.to_bf16_bits(f)
    return scene


def test_noalloc_matches_gs_render_on_calls_in_a_row(gsr):
    scene = _scene()
    cams = [synth.camera(240, 136, 175.0), synth.camera(200, 120, 150.0), synth.camera(240, 136, 175.0)]
    poses = [synth.look_pose((100.0, 40.0, 60.0), 0.0, 0.5), synth.look_pose((90.0, 70.0, 70.0), 1.0, 0.3),
             synth.look_pose((100.0, 40.0, 60.0), 0.0, 0.5)]
    S = gsr.Scene(scene)
    keep = []
    desc = _device_desc(gsr, scene, keep)
    stream = torch.cuda.current_stream().cuda_stream
    # larger view, smaller view, then the larger one again: stale tile counts and
    # pairs of either size must not leak into the next call
    for cam, T in zip(cams, poses):
        ref = S.render(cam, T)
        out = {k: torch.full_like(v, 7) for k, v in ref.items()}
        gsr.gs_render_noalloc(desc, gsr.camera(cam), gsr.pose(T), S.outputs_struct(out), stream)
        torch.cuda.synchronize()
        for k in ref:  # same kernels, same inputs: identical bits
            torch.testing.assert_close(out[k], ref[k], rtol=0, atol=0, msg=k)
    S.close()


def test_noalloc_rejects_sizes_beyond_its_limits(gsr):
    keep = []
    big = synth.tiny_scene(1, n=gsr.GS_NOALLOC_MAX_GAUSSIANS + 1)
    desc = _device_desc(gsr, big, keep)
    out = gsr.Scene.alloc_outputs(synth.tiny_camera())
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(gsr.GsError) as e:
        gsr.gs_render_noalloc(desc, gsr.camera(synth.tiny_camera()), gsr.pose(np.eye(4)),
                              gsr.Scene.outputs_struct(out), stream)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG and "32768" in str(e.value)
    small = _device_desc(gsr, synth.tiny_scene(2, n=100), keep)
    huge_cam = synth.camera(4096, 4096, 1000.0)
    with pytest.raises(gsr.GsError) as e:
        gsr.gs_render_noalloc(small, gsr.camera(huge_cam), gsr.pose(np.eye(4)), gsr.gs_outputs(), stream)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG and "tiles" in str(e.value)
