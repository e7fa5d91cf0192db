"""Pins of the oracle's projection / footprint layer against closed forms.

Algorithm 1 of the paper fixes the projection (world -> camera by T, depth =
camera z, perspective division, then K; Eq. 10 pi([x,y,z]) = [x/z, y/z]). The
EWA footprint constants (0.3 px dilation, 1.3 guard, 0.1 eigenvalue floor,
3 sigma, 16 px tiles, near plane 0.2) are this project's readings; the values
below are worked out by hand from them.
"""
import math

import numpy as np
import pytest

from paper_2507_15683_gb300 import synth
from tests.oracle_scenes import cam, rot_z


def _proj(O, means, scales=None, quats=None, c=None, T=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    scales = np.full((n, 3), 0.1, np.float32) if scales is None else np.asarray(scales, np.float32).reshape(n, 3)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    cov = O.cov3d_f32(scales, quats)
    return O.project_f32(means, cov, c or cam(), np.eye(4) if T is None else T)


def test_alg1_identity_pose_exact_points(oracle):
    # fx = fy = 128, cx = cy = 64: every value below is exact in binary32
    c = cam(128, 128, 128.0)
    ri, rf = _proj(oracle, [[0, 0, 5], [1, 0, 4], [-2, 1, 8]], c=c)
    np.testing.assert_array_equal(rf[:, oracle.F_Z], [5, 4, 8])
    np.testing.assert_array_equal(rf[:, oracle.F_U], [64, 96, 32])
    np.testing.assert_array_equal(rf[:, oracle.F_V], [64, 64, 80])


def test_alg1_rotated_pose_boresight(oracle):
    # aerial camera: a point on the optical axis lands on the principal point,
    # a point half a focal length to the right lands at cx + fx / 2
    T = synth.aerial_pose()
    R = T[:3, :3]
    c_w = -R.T @ T[:3, 3]
    fwd, right, down = R[2], R[0], R[1]
    d = 300.0 / math.cos(math.radians(30))
    pts = np.stack([c_w + d * fwd, c_w + d * (fwd + 0.5 * right), c_w + d * (fwd - 0.25 * down)])
    c = synth.aerial_camera()
    ri, rf = _proj(oracle, pts, c=c, T=T)
    np.testing.assert_allclose(rf[:, oracle.F_U], [960, 960 + 700, 960], atol=2e-3)
    np.testing.assert_allclose(rf[:, oracle.F_V], [540, 540, 540 - 350], atol=2e-3)
    np.testing.assert_allclose(rf[:, oracle.F_Z], d, rtol=1e-6)


def test_near_plane(oracle):
    ri, rf = _proj(oracle, [[0, 0, 0.19], [0, 0, 0.2], [0, 0, -3.0]], scales=np.full((3, 3), 1e-3))
    assert list(ri[:, oracle.I_STATUS]) == [oracle.CULL_NEAR, oracle.VISIBLE, oracle.CULL_NEAR]


def test_footprint_isotropic_on_axis(oracle):
    # s = 0.1, z = 5, f = 100: J s = 2 px -> Sigma' = diag(4.3, 4.3); equal eigenvalues
    # leave the 0.1 floor under the discriminant: lambda = 4.3 + sqrt(0.1), r = ceil(3 sqrt(lambda)) = 7
    ri, rf = _proj(oracle, [[0, 0, 5]])
    assert rf[0, oracle.F_A] == pytest.approx(4.3, rel=1e-6)
    assert rf[0, oracle.F_C] == pytest.approx(4.3, rel=1e-6)
    assert abs(rf[0, oracle.F_B]) < 1e-6
    lam = 4.3 + math.sqrt(0.1)
    assert rf[0, oracle.F_R] == math.ceil(3 * math.sqrt(lam)) == 7
    # centre 64 +- 7 -> tiles 3..4 in x and y
    assert list(ri[0, 1:]) == [3, 4, 3, 4, 4]


def test_footprint_anisotropic_quaternion(oracle):
    # quaternion = 90 deg about z maps the local x axis to world y:
    # world Sigma = diag(0.05^2, 0.2^2, 0.1^2); on axis at z = 5, f = 100 -> (J s)^2 = 400 s^2
    q = [[math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]]
    ri, rf = _proj(oracle, [[0, 0, 5]], scales=[[0.2, 0.05, 0.1]], quats=q)
    assert rf[0, oracle.F_A] == pytest.approx(400 * 0.05 ** 2 + 0.3, rel=1e-5)
    assert rf[0, oracle.F_C] == pytest.approx(400 * 0.2 ** 2 + 0.3, rel=1e-5)
    assert abs(rf[0, oracle.F_B]) < 1e-5
    # a larger eigenvalue 16.3 with a large discriminant: r = ceil(3 sqrt(16.3))
    assert rf[0, oracle.F_R] == math.ceil(3 * math.sqrt(16.3))


def test_footprint_camera_roll(oracle):
    # rolling the camera 90 deg about its axis swaps the footprint's axes
    ri0, rf0 = _proj(oracle, [[0, 0, 5]], scales=[[0.2, 0.05, 0.1]])
    ri1, rf1 = _proj(oracle, [[0, 0, 5]], scales=[[0.2, 0.05, 0.1]], T=rot_z(90))
    assert rf0[0, oracle.F_A] == pytest.approx(400 * 0.2 ** 2 + 0.3, rel=1e-5)
    assert rf1[0, oracle.F_A] == pytest.approx(rf0[0, oracle.F_C], rel=1e-5)
    assert rf1[0, oracle.F_C] == pytest.approx(rf0[0, oracle.F_A], rel=1e-5)


def test_isotropic_footprint_independent_of_rotation(oracle):
    g = np.random.default_rng(5)
    q = g.standard_normal((64, 4)).astype(np.float32)
    means = np.tile(np.array([[0.3, -0.2, 5.0]], np.float32), (64, 1))
    ri, rf = _proj(oracle, means, scales=np.full((64, 3), 0.07), quats=q)
    for k in (oracle.F_A, oracle.F_B, oracle.F_C):
        np.testing.assert_allclose(rf[:, k], rf[0, k], rtol=2e-5, atol=2e-6)


def test_off_axis_jacobian_and_guard(oracle):
    # point (x, 0, z): Sigma' = s^2 (f/z)^2 (1 + xhat^2/z^2) + 0.3 along x, xhat clamped at 1.3 tan(fov/2)
    s, z, f = 0.1, 5.0, 100.0
    lim = 1.3 * (0.5 * 128 / f)
    ri, rf = _proj(oracle, [[0.3 * z, 0, z], [2.0 * z, 0, z]], scales=np.full((2, 3), s))
    base = (s * f / z) ** 2
    assert rf[0, oracle.F_A] == pytest.approx(base * (1 + 0.3 ** 2) + 0.3, rel=1e-5)
    assert rf[1, oracle.F_A] == pytest.approx(base * (1 + lim ** 2) + 0.3, rel=1e-5)
    assert rf[0, oracle.F_C] == pytest.approx(base + 0.3, rel=1e-5)


def test_tile_rect_against_interval_enumeration(oracle):
    # a tile (16 px, half open) is kept iff it meets the closed square [u-r, u+r] x [v-r, v+r]
    sc = synth.tiny_scene(7, n=3000)
    sc["means"][:, :2] *= 1.5  # many Gaussians straddle the image border
    c = cam(100, 75, 90.0, 50.0, 37.5)
    cov = oracle.cov3d_f32(sc["scales"], sc["quats"])
    ri, rf = oracle.project_f32(sc["means"], cov, c, np.eye(4))
    tx, ty = oracle.tiles_of(c)
    n_checked = 0
    for i in range(ri.shape[0]):
        st = ri[i, oracle.I_STATUS]
        if st not in (oracle.VISIBLE, oracle.CULL_EMPTY):
            continue
        u, v, r = float(rf[i, oracle.F_U]), float(rf[i, oracle.F_V]), float(rf[i, oracle.F_R])
        xs = [t for t in range(tx) if 16 * t <= u + r and u - r < 16 * t + 16]
        ys = [t for t in range(ty) if 16 * t <= v + r and v - r < 16 * t + 16]
        if st == oracle.CULL_EMPTY:
            assert not xs or not ys
            continue
        assert (min(xs), max(xs), min(ys), max(ys)) == tuple(ri[i, 1:5])
        assert len(xs) * len(ys) == ri[i, oracle.I_COUNT]
        n_checked += 1
    assert n_checked > 500


def test_binary32_layer_close_to_binary64(oracle):
    # the binary32 centre must agree with a binary64 evaluation of Algorithm 1
    sc = synth.aerial_scene(11, 20000)
    c = synth.aerial_camera()
    T = synth.aerial_pose()
    cov = oracle.cov3d_f32(sc["scales"], sc["quats"])
    ri, rf = oracle.project_f32(sc["means"], cov, c, T)
    p = sc["means"].astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    u = c["fx"] * p[:, 0] / p[:, 2] + c["cx"]
    vis = ri[:, 0] == oracle.VISIBLE
    assert vis.sum() > 1000
    np.testing.assert_allclose(rf[vis, oracle.F_U], u[vis], atol=5e-3)
    np.testing.assert_allclose(rf[vis, oracle.F_Z], p[vis, 2], rtol=1e-6)


def test_binning_order_and_ranges(oracle):
    sc = synth.tiny_scene(0)
    c = synth.tiny_camera()
    cov = oracle.cov3d_f32(sc["scales"], sc["quats"])
    ri, rf = oracle.project_f32(sc["means"], cov, c, np.eye(4))
    ts, keys, gids = oracle.bin_tiles(ri, rf, c)
    assert ts[-1] == len(keys) == ri[ri[:, 0] == 0, oracle.I_COUNT].sum()
    # keys are strictly increasing as (tile, depth bits, index)
    composite = [(int(k) >> 32, int(k) & 0xFFFFFFFF, int(g)) for k, g in zip(keys, gids)]
    assert composite == sorted(composite)
    assert len(set(composite)) == len(composite)
    zb = rf[:, oracle.F_Z].view(np.uint32)
    for t in range(len(ts) - 1):
        seg = slice(ts[t], ts[t + 1])
        assert np.all((keys[seg] >> np.uint64(32)) == t)
        assert np.all((keys[seg] & np.uint64(0xFFFFFFFF)) == zb[gids[seg]])
