"""Small hand-built scenes for the oracle pins (plain data, no method arithmetic)."""
import math

import numpy as np


def scene_of(means, scales, quats=None, opacities=None, dc=None, sh_degree=0, sh_rest=None, feats_bf16=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    scales = np.asarray(scales, np.float32).reshape(n, 3)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else \
        np.asarray(quats, np.float32).reshape(n, 4)
    opacities = np.full(n, 0.5, np.float32) if opacities is None else np.asarray(opacities, np.float32).reshape(n)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    if dc is not None:
        sh[:, 0, :] = np.asarray(dc, np.float32).reshape(n, 3)
    if sh_rest is not None:
        sh[:, 1:, :] = sh_rest
    return {"means": means, "scales": scales, "quats": quats, "opacities": opacities, "sh": sh,
            "sh_degree": sh_degree, "feats_bf16": feats_bf16}


def cam(w=128, h=128, f=100.0, cx=64.0, cy=64.0):
    return {"width": w, "height": h, "fx": f, "fy": f, "cx": cx, "cy": cy}


def rot_z(deg):
    a = math.radians(deg)
    R = np.eye(4)
    R[:2, :2] = [[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]]
    return R


Y00 = 1.0 / (2.0 * math.sqrt(math.pi))
