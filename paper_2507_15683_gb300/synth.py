"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras and poses.

This module only draws inputs. It holds none of the rasterizer's arithmetic
and is the one module that both the CUDA path's tests/benchmark and the CPU
oracle consume. Random numbers come from numpy's counter-based Philox bit
generator, seeded per workload.

Workloads (shapes from the paper's remote-sensing scenes: ~1 km^2 areas seen
from a few hundred metres at 1920x1080, Table 1 of the paper):

* ``tiny``      1,000 Gaussians in front of an identity camera, SH degree 0,
                128x128, fx=fy=128.
* ``aerial``    1,000,000 Gaussians over 1 km x 1 km (95 % ground, 5 % in 500
                building clusters up to 60 m), SH degree 3, 1920x1080, f=1400,
                camera at (500, 200, 300) m pitched 30 deg from nadir toward +y.
* ``refine``    500,000 Gaussians drawn like ``aerial`` over 1000 x 500 m, 960x540
                (f=700); the query pose is the reference pose perturbed by 2 deg
                about a random axis and 5 m in a random direction.
* ``batched``   2,000,000 Gaussians in 4 quadrant partitions of 500k, SH degree 3
                plus 32 BF16 feature channels (N(0,1), L2-normalised); 84 poses
                (64 @ 480x270, 16 @ 960x540, 4 @ 1920x1080) inside a 200 m disc
                at 200-400 m altitude, yaw U(0, 2 pi), pitch U(0, 45) deg.
* ``large``     6,000,000 Gaussians in a 4 x 4 grid of 500 m cells, SH degree 3
                plus 32 BF16 features; 8 poses, pyramid 480x270 .. 3840x2160.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def camera(width: int, height: int, f: float, cx: float | None = None, cy: float | None = None) -> dict:
    return {"width": int(width), "height": int(height), "fx": float(f), "fy": float(f),
            "cx": float(width / 2 if cx is None else cx), "cy": float(height / 2 if cy is None else cy)}


def look_pose(centre, yaw: float, pitch_from_nadir: float) -> np.ndarray:
    """World-to-camera 4x4 (x right, y down, z forward) for a camera at ``centre``
    heading ``yaw`` (0 = +y, world z up) and tilted ``pitch_from_nadir`` rad."""
    h = np.array([math.sin(yaw), math.cos(yaw), 0.0])
    fwd = math.cos(pitch_from_nadir) * np.array([0.0, 0.0, -1.0]) + math.sin(pitch_from_nadir) * h
    right = np.array([math.cos(yaw), -math.sin(yaw), 0.0])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = -R @ np.asarray(centre, np.float64)
    return T


def _rot_axis_angle(axis, ang):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def perturb_pose(T, g: np.random.Generator, rot_deg: float, trans_m: float) -> np.ndarray:
    """Rotate the camera by ``rot_deg`` about a uniform random axis (about its
    own centre) and move its centre ``trans_m`` in a uniform random direction."""
    T = np.asarray(T, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    c = -R.T @ t
    ax = g.standard_normal(3)
    dr = g.standard_normal(3)
    dr = dr / np.linalg.norm(dr)
    R2 = _rot_axis_angle(ax, math.radians(rot_deg)) @ R
    c2 = c + trans_m * dr
    out = np.eye(4)
    out[:3, :3] = R2
    out[:3, 3] = -R2 @ c2
    return out


def _random_quats(g, n):
    q = g.standard_normal((n, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sigmoid(x):
    return (1.0 / (1.0 + np.exp(-x))).astype(np.float32)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest even) and return the bit patterns."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


def tiny_scene(seed: int = 0, n: int = 1000, sh_degree: int = 0) -> dict:
    g = rng(seed)
    means = np.empty((n, 3), np.float32)
    means[:, 0] = g.uniform(-2, 2, n)
    means[:, 1] = g.uniform(-2, 2, n)
    means[:, 2] = g.uniform(4, 8, n)
    scales = np.exp(g.normal(-3.0, 0.5, (n, 3))).astype(np.float32)
    quats = _random_quats(g, n)
    opac = _sigmoid(g.standard_normal(n))
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = g.uniform(0, 1, (n, 3))
    if K > 1:
        sh[:, 1:, :] = g.normal(0, 0.05, (n, K - 1, 3))
    return {"means": means, "scales": scales, "quats": quats, "opacities": opac, "sh": sh,
            "sh_degree": sh_degree, "feats_bf16": None}


def tiny_camera() -> dict:
    return camera(128, 128, 128.0, 64.0, 64.0)


def aerial_scene(seed: int, n: int, extent=(0.0, 1000.0, 0.0, 1000.0), n_clusters: int | None = None,
                 sh_degree: int = 3, feat_dim: int = 0, building_frac: float = 0.05,
                 keep_f32: bool = False) -> dict:
    """Ground plane (z ~ N(0, 20 m)) plus clustered 'building' Gaussians.
    keep_f32 also returns the unrounded binary32 features ("feats_f32")."""
    g = rng(seed)
    x0, x1, y0, y1 = extent
    nb = int(round(n * building_frac))
    ng = n - nb
    if n_clusters is None:
        n_clusters = max(1, int(round(500 * (x1 - x0) * (y1 - y0) / 1e6)))
    means = np.empty((n, 3), np.float32)
    means[:ng, 0] = g.uniform(x0, x1, ng)
    means[:ng, 1] = g.uniform(y0, y1, ng)
    means[:ng, 2] = g.normal(0.0, 20.0, ng)
    cc = np.stack([g.uniform(x0, x1, n_clusters), g.uniform(y0, y1, n_clusters)], 1)
    which = g.integers(0, n_clusters, nb)
    means[ng:, 0:2] = cc[which] + g.normal(0.0, 5.0, (nb, 2))
    means[ng:, 2] = g.uniform(0.0, 60.0, nb)
    scales = np.exp(g.normal(math.log(0.5), 0.7, (n, 3))).astype(np.float32)
    quats = _random_quats(g, n)
    opac = _sigmoid(g.normal(1.0, 1.5, n))
    K = (sh_degree + 1) ** 2
    sh = np.empty((n, K, 3), np.float32)
    sh[:, 0, :] = g.uniform(0, 1, (n, 3))
    if K > 1:
        sh[:, 1:, :] = g.normal(0, 0.05, (n, K - 1, 3))
    feats = None
    if feat_dim:
        f = g.standard_normal((n, feat_dim)).astype(np.float32)
        f /= np.linalg.norm(f, axis=1, keepdims=True)
        feats = to_bf16_bits(f)
    out = {"means": means, "scales": scales, "quats": quats, "opacities": opac, "sh": sh,
           "sh_degree": sh_degree, "feats_bf16": feats}
    if keep_f32 and feat_dim:
        out["feats_f32"] = f
    return out


def aerial_camera(width=1920, height=1080, f=1400.0) -> dict:
    return camera(width, height, f)


def aerial_pose() -> np.ndarray:
    return look_pose((500.0, 200.0, 300.0), 0.0, math.radians(30.0))


def refine_workload(seed: int = 3, n: int = 500_000):
    """Scene, camera, reference pose and perturbed query pose for pose refinement."""
    scene = aerial_scene(seed, n, extent=(0.0, 1000.0, 150.0, 650.0))
    cam = aerial_camera(960, 540, 700.0)
    T_gt = aerial_pose()
    T_q = perturb_pose(T_gt, rng(seed + 1000), 2.0, 5.0)
    return scene, cam, T_gt, T_q


def partitioned_scene(seed: int, cells_x: int, cells_y: int, per_cell: int, cell_m: float = 500.0,
                      sh_degree: int = 3, feat_dim: int = 32, keep_f32: bool = False) -> dict:
    """Scene made of a grid of square cells; Gaussians are stored cell by cell
    and ``partition_offsets`` gives each cell's index range."""
    parts = []
    for cy in range(cells_y):
        for cx in range(cells_x):
            parts.append(aerial_scene(seed * 1000 + cy * cells_x + cx, per_cell,
                                      extent=(cx * cell_m, (cx + 1) * cell_m, cy * cell_m, (cy + 1) * cell_m),
                                      sh_degree=sh_degree, feat_dim=feat_dim, keep_f32=keep_f32))
    out = {k: np.concatenate([p[k] for p in parts]) for k in ("means", "scales", "quats", "opacities", "sh")}
    out["feats_bf16"] = np.concatenate([p["feats_bf16"] for p in parts]) if feat_dim else None
    if keep_f32 and feat_dim:
        out["feats_f32"] = np.concatenate([p["feats_f32"] for p in parts])
    out["sh_degree"] = sh_degree
    out["partition_offsets"] = np.arange(0, per_cell * len(parts) + 1, per_cell, dtype=np.int64)
    return out


def batched_views(seed: int = 4, centre=(500.0, 500.0), radius=200.0, counts=(64, 16, 4),
                  sizes=((480, 270, 350.0), (960, 540, 700.0), (1920, 1080, 1400.0))):
    """Candidate poses and cameras of mixed resolution."""
    g = rng(seed)
    cams, poses = [], []
    for cnt, (w, h, f) in zip(counts, sizes):
        for _ in range(cnt):
            r = radius * math.sqrt(g.uniform(0, 1))
            th = g.uniform(0, 2 * math.pi)
            c = (centre[0] + r * math.cos(th), centre[1] + r * math.sin(th), g.uniform(200, 400))
            poses.append(look_pose(c, g.uniform(0, 2 * math.pi), math.radians(g.uniform(0, 45))))
            cams.append(camera(w, h, f))
    return cams, poses
