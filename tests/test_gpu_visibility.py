"""GPU render-gradient visibility check (Sec. 3.2, Algorithm 1) against the
oracle, through the C ABI (gs_visibility).

Per Gaussian the oracle gives M^r (binary64 forward-mode gradient of the
summed colours along its mean is non-zero), M^i (projected centre inside the
image) and M = M^r and M^i, plus a flag for decisions within rounding. On every
unflagged Gaussian the three bits must be identical; the projected centre must
agree to 1e-3 px (plus 1e-6 of its magnitude); the mean gradient to the fp32
tolerance below. Over all Gaussians, whatever the oracle evaluated, the
outputs must be consistent with one another (M = M^r and M^i, M^r exactly
where the gradient is non-zero, M^i exactly where (U, V) is inside, the
compacted list is the ascending list of M with its (U, V)).
"""
import math

import numpy as np
import pytest
import torch

from paper_2507_15683_gb300 import synth
from tests.oracle_scenes import scene_of

pytestmark = pytest.mark.gpu

# fp32 mean gradient vs binary64: the reverse pass sums per-pixel terms
# e dx^k dy^l whose total cancels strongly (moving an unoccluded Gaussian
# across the image changes the summed colour only at its footprint's cut-off),
# so the error is bounded relative to the largest gradient of the view rather
# than to each Gaussian's own.
GRAD_REL = 2e-4
GRAD_ABS_OF_MAX = 2e-6


def _gpu(gsr, scene, cam, T, **kw):
    S = gsr.Scene(scene, **kw)
    r = S.visibility(cam, T)
    r2 = S.visibility(cam, T)  # a second call: same decisions
    S.close()
    out = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    np.testing.assert_array_equal(r2["mask"].cpu().numpy(), out["mask"])
    return out


def _consistent(g, cam):
    """Relations between the outputs that hold exactly, for every Gaussian."""
    m = g["mask"]
    M, Mr, Mi = (m & 1) != 0, (m & 2) != 0, (m & 4) != 0
    assert not np.any(m & ~np.uint8(7))
    np.testing.assert_array_equal(M, Mr & Mi)
    np.testing.assert_array_equal(Mr, np.any(g["grad"] != 0, axis=1))
    u, v = g["uv"][:, 0], g["uv"][:, 1]
    np.testing.assert_array_equal(Mi, (u >= 0) & (u < cam["width"]) & (v >= 0) & (v < cam["height"]))
    ids = np.nonzero(M)[0]
    assert g["n_visible"] == len(ids)
    np.testing.assert_array_equal(g["ids"], ids)
    np.testing.assert_array_equal(g["uv_visible"], g["uv"][ids])
    return M, Mr, Mi


def _check(g, o, min_ok=0.95):
    gids = o["gids"]
    m = g["mask"][gids]
    M, Mr, Mi = (m & 1) != 0, (m & 2) != 0, (m & 4) != 0
    ok = ~o["flag"]
    assert ok.mean() >= min_ok
    np.testing.assert_array_equal(Mi[ok], o["M_i"][ok])
    np.testing.assert_array_equal(Mr[ok], o["M_r"][ok])
    np.testing.assert_array_equal(M[ok], o["M"][ok])
    fin = np.all(np.isfinite(o["uv"]), axis=1)
    du = np.abs(g["uv"][gids][fin] - o["uv"][fin])
    assert np.all(du <= 1e-3 + 1e-6 * np.abs(o["uv"][fin])), du.max()
    big = np.linalg.norm(o["grad"], axis=1).max()
    err = np.linalg.norm(g["grad"][gids].astype(np.float64) - o["grad"], axis=1)
    lim = GRAD_REL * np.linalg.norm(o["grad"], axis=1) + GRAD_ABS_OF_MAX * big
    print("visibility: %d checked, %d flagged, %d kept; grad err max %.3g (of max norm %.3g), worst ratio %.3g"
          % (len(gids), (~ok).sum(), int(o["M"].sum()), err.max(), big, (err / lim).max()))
    assert np.all(err <= lim)


def test_visibility_tiny_scene(oracle, gsr):
    sc = synth.tiny_scene(11, n=400, sh_degree=1)
    sc["sh"][:, 1:, :] *= 3.0
    cam = synth.tiny_camera()
    T = synth.perturb_pose(np.eye(4), synth.rng(12), 3.0, 0.1)
    o = oracle.visibility(sc, cam, T, n_threads=16)
    g = _gpu(gsr, sc, cam, T)
    _consistent(g, cam)
    _check(g, o)
    assert 0 < g["n_visible"] < len(sc["means"])
    # the reverse pass walks back through exactly the pairs the render blended:
    # the oracle's per-pixel blend counts, up to pixels with a near-tie decision
    S = gsr.Scene(sc)
    S.visibility(cam, T)
    blended, evaluated = gsr.gs_scene_work_counts(S.handle)
    S.close()
    r = oracle.render(sc, cam, T, geom64=True)
    ok = (r["flags"] & oracle.TIE_IMAGE) == 0
    assert abs(blended - int(r["n_blend"].sum())) <= int(r["n_blend"][~ok].sum())
    assert evaluated >= blended > 0


def test_visibility_structural_cases(oracle, gsr):
    cam = synth.camera(128, 128, 100.0)
    # three walls in front (opacity 0.985) saturate the transmittance before a small
    # Gaussian behind them is reached; a fifth projects left of the image but reaches in;
    # a sixth lies behind the camera
    means = [[0, 0, 5.0], [0, 0, 5.5], [0, 0, 6.0], [0.01, 0.01, 8.0], [-3.3, 0.0, 5.0], [0.0, 0.0, -4.0]]
    scales = [[10.0] * 3, [10.0] * 3, [10.0] * 3, [0.02] * 3, [0.3] * 3, [0.5] * 3]
    sc = scene_of(means, scales, opacities=[0.985, 0.985, 0.985, 0.9, 0.9, 0.9],
                  dc=[[0.5, 0.1, 0.1], [0.1, 0.5, 0.1], [0.1, 0.1, 0.5], [0.9, 0.9, 0.9], [0.2, 0.8, 0.2],
                      [0.5, 0.5, 0.5]])
    o = oracle.visibility(sc, cam, np.eye(4))
    g = _gpu(gsr, sc, cam, np.eye(4))
    M, Mr, Mi = _consistent(g, cam)
    _check(g, o, min_ok=1.0)
    assert M[0] and M[1] and not Mr[3] and Mi[3] and Mr[4] and not Mi[4] and not Mr[5]
    assert g["uv"][4, 0] < 0


def test_visibility_exact_image_edges(oracle, gsr):
    """Algorithm 1's half-open image: centres projected exactly onto the left and
    top edges are in, exactly onto the right and bottom edges are out (16 x 16
    image, f = c = 8, z = 1: x = -1 gives u = 0, x = 1 gives u = 16)."""
    cam = {"width": 16, "height": 16, "fx": 8.0, "fy": 8.0, "cx": 8.0, "cy": 8.0}
    means = [[-1.0, 0.0, 1.0], [1.0, 0.0, 1.0], [0.0, -1.0, 1.0], [0.0, 1.0, 1.0]]
    sc = scene_of(means, [[0.05] * 3] * 4, opacities=[0.9] * 4, dc=[[0.5, 0.5, 0.5]] * 4)
    o = oracle.visibility(sc, cam, np.eye(4), want_grad=False)
    g = _gpu(gsr, sc, cam, np.eye(4))
    _consistent(g, cam)
    np.testing.assert_array_equal(g["uv"], [[0.0, 8.0], [16.0, 8.0], [8.0, 0.0], [8.0, 16.0]])
    np.testing.assert_array_equal((g["mask"] & 4) != 0, o["M_i"])
    assert list(o["M_i"]) == [True, False, True, False]


def test_visibility_small_aerial(oracle, gsr):
    """240 x 136 (15 x 9 tiles, ragged last row), 20,000 Gaussians, view-dependent
    colour: every Gaussian's M^i, and M^r / gradient of every Gaussian without a
    tile rectangle plus 400 sampled among those with one."""
    sc = synth.aerial_scene(41, 20000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20)
    sc["sh"][:, 1:, :] *= 3.0
    cam = synth.camera(240, 136, 175.0)
    T = synth.perturb_pose(synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0)), synth.rng(3), 1.0, 1.0)
    cov = oracle.cov3d_f32(sc["scales"], sc["quats"])
    ri, _ = oracle.project_f32(sc["means"], cov, cam, T)
    has_rect = ri[:, oracle.I_STATUS] == oracle.VISIBLE
    sample = synth.rng(4).choice(np.nonzero(has_rect)[0], 400, replace=False)
    gids = np.sort(np.concatenate([np.nonzero(~has_rect)[0], sample]))
    o = oracle.visibility(sc, cam, T, n_threads=16, gids=gids)
    g = _gpu(gsr, sc, cam, T)
    _consistent(g, cam)
    _check(g, o)
    assert not np.any(g["mask"][~has_rect] & 2)  # no tile, no gradient


def test_visibility_streamed_partitions_equal_resident(gsr):
    """A streamed scene is made resident for the in-image test: the same masks as
    the resident scene, including partitions no pixel sees."""
    sc = synth.partitioned_scene(5, 3, 3, 4000, cell_m=120.0)
    cam = synth.camera(320, 180, 250.0)
    T = synth.look_pose((60.0, 60.0, 80.0), 0.3, math.radians(20.0))
    a = _gpu(gsr, sc, cam, T)
    b = _gpu(gsr, sc, cam, T, stream_partitions=True)
    _consistent(a, cam)
    _consistent(b, cam)
    np.testing.assert_array_equal(a["mask"], b["mask"])
    np.testing.assert_array_equal(a["uv"], b["uv"])


def test_visibility_empty_and_arguments(gsr):
    sc = scene_of(np.zeros((0, 3)), np.zeros((0, 3)))
    cam = synth.camera(64, 48, 50.0)
    S = gsr.Scene(sc)
    r = S.visibility(cam, np.eye(4))
    assert r["n_visible"] == 0 and r["mask"].numel() == 0
    with pytest.raises(gsr.GsError) as e:
        gsr.gs_visibility(S.handle, gsr.camera(cam), gsr.pose(np.eye(4)), 0, None, None, None, None,
                          gsr._stream())
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    S.close()


def test_visibility_full_size_1080p(oracle, gsr):
    """1,000,000 Gaussians at 1920 x 1080 (the render workload): the exact output
    relations for every Gaussian, every Gaussian's M^i against the oracle's
    projection, and M^r / gradient of 48 sampled Gaussians with a tile rectangle."""
    sc = synth.aerial_scene(2, 1_000_000)
    cam = synth.aerial_camera()
    T = synth.perturb_pose(synth.aerial_pose(), synth.rng(100), 2.0, 5.0)
    g = _gpu(gsr, sc, cam, T)
    _consistent(g, cam)
    cov = oracle.cov3d_f32(sc["scales"], sc["quats"])
    ri, _ = oracle.project_f32(sc["means"], cov, cam, T)
    has_rect = ri[:, oracle.I_STATUS] == oracle.VISIBLE
    assert not np.any(g["mask"][~has_rect] & 2)
    sample = np.sort(synth.rng(7).choice(np.nonzero(has_rect)[0], 48, replace=False))
    o = oracle.visibility(sc, cam, T, n_threads=16, gids=sample)
    _check(g, o, min_ok=0.9)
    # M^i and (U, V) of every Gaussian (projection only: no gradient evaluated)
    oi = oracle.visibility(sc, cam, T, want_grad=False)
    ok = ~oi["flag"]
    np.testing.assert_array_equal((g["mask"][ok] & 4) != 0, oi["M_i"][ok])
    fin = np.all(np.isfinite(oi["uv"]), axis=1)
    assert np.all(np.abs(g["uv"][fin] - oi["uv"][fin]) <= 1e-3 + 1e-6 * np.abs(oi["uv"][fin]))
