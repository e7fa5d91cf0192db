"""Dense render-and-match rounds and Algorithm 2's pose consistency check --
fp64 oracle (Sec. 3.4, Algorithm 2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg of
``bench.py``, never by the product path.

One round renders the feature map, depth and alpha at the current pose (the
oracle renderer), matches the query features against them coarse to fine
(``oracle.pmm``, Eq. 11) and solves Eq. 10 on the fine matches
(``oracle.pnp``); its pose starts the next round. Algorithm 2 then compares
consecutive rounds with Psi (``oracle.pose_diff``: trace-clamped angle of
R1 R2^T, distance of the translation columns) and calls the result
unreliable when an angle exceeds the threshold.

Readings (the same in the CUDA path): Psi is evaluated for every consecutive
pair (T_i, T_i+1) -- the listing names (T_1, T_2) in each iteration; every
round runs before the check; the translation distance is reported only.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from oracle import pmm as PM
from oracle import pnp as OP


def consistency(poses, max_angle_deg=20.0):
    """Algorithm 2 on a list of poses: (reliable, angles, translation distances)."""
    ang, tr = [], []
    for a, b in zip(poses[:-1], poses[1:]):
        t, d = O.pose_diff(a, b)
        ang.append(t)
        tr.append(d)
    return all(t <= max_angle_deg for t in ang), ang, tr


def dense_round(scene, cam, T, feat_query, words, pmm_tau=PM.TAU, tau=2.0, min_alpha=OP.MIN_ALPHA,
                refine_iters=5, n_threads=16):
    """One render -> PMM -> PnP round from pose T. Returns (pose, fine matches, pnp record)."""
    H, W = int(cam["height"]), int(cam["width"])
    r = O.render(scene, cam, T, geom64=True, n_threads=n_threads)
    Fr = np.ascontiguousarray(r["feats"].T.reshape(32, H, W).astype(np.float32))
    coarse = PM.coarse_pmm(feat_query, Fr, pmm_tau)
    fine = PM.fine_pmm(feat_query, Fr, coarse["matches"], pmm_tau)
    depth = r["depth"].reshape(H, W).astype(np.float32)
    alpha = r["alpha"].reshape(H, W).astype(np.float32)
    res = OP.pnp_ransac(depth, alpha, cam, T, fine["matches"], words, tau, refine_iters, min_alpha)
    return res["T"], fine, res


def localize(scene, cam, T_init, feat_query, words, n_rounds=3, max_angle_deg=20.0, **kw):
    """n rounds then Algorithm 2. words: (n_rounds, n_hypotheses, 3) uint32.
    Returns dict: T (last round), reliable, round_T, angle_deg, trans, rounds."""
    T = np.asarray(T_init, np.float64)
    poses, rounds = [], []
    for i in range(n_rounds):
        T, fine, res = dense_round(scene, cam, T, feat_query, words[i], **kw)
        poses.append(T)
        rounds.append({"fine": fine, "pnp": res})
    ok, ang, tr = consistency(poses, max_angle_deg)
    return {"T": poses[-1], "reliable": ok, "round_T": poses, "angle_deg": ang, "trans": tr, "rounds": rounds}
