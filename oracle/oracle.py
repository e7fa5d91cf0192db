"""ctypes/numpy front end of the CPU oracle (gs_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``. The
product path (``paper_2507_15683_gb300``) never imports it, and it imports
nothing from the product except the seeded input generators' plain data.

Every function documents the passage of the paper it follows (Hi^2-GSLoc,
arXiv 2507.15683): Sec. 3.1 (Gaussian primitive, alpha blending of colour and
features), Algorithm 1 (projection), Eq. 10 (pinhole projection), Algorithm 2
(pose difference). The rest are the project's stated readings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16
ALPHA_FLOOR = 1.0 / 255.0
ALPHA_CAP = 0.99
T_CUTOFF = 1e-4

VISIBLE, CULL_NEAR, CULL_DET, CULL_RADIUS, CULL_EMPTY = range(5)
I_STATUS, I_X0, I_X1, I_Y0, I_Y1, I_COUNT = range(6)
F_Z, F_U, F_V, F_A, F_B, F_C, F_DET, F_R = range(8)
TIE_POWER, TIE_ALPHA_FLOOR, TIE_T_CUTOFF, TIE_ALPHA_CAP = 1, 2, 4, 8
TIE_RGB_CLAMP, TIE_J_CLAMP, TIE_RESIDUAL = 16, 32, 64
TIE_IMAGE = TIE_POWER | TIE_ALPHA_FLOOR | TIE_T_CUTOFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE binary32, no FP contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "gs_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int), ("feat_dim", ctypes.c_int),
                ("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("feats_bf16", ctypes.c_void_p),
                ("feats_f32", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("geom64", ctypes.c_int), ("want_grad", ctypes.c_int), ("n_threads", ctypes.c_int),
                ("pixels", ctypes.c_void_p), ("n_pixels", ctypes.c_int64),
                ("target_rgb", ctypes.c_void_p), ("target_depth", ctypes.c_void_p),
                ("pixel_weight", ctypes.c_void_p), ("depth_weight", ctypes.c_double),
                ("tie_rel", ctypes.c_double), ("tie_rel_T", ctypes.c_double),
                ("mean_tangent_gid", ctypes.c_int64)]


class _Out(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("rgb", "depth", "alpha", "final_T", "last_idx", "n_eval", "n_blend", "flags", "feats",
                 "loss", "grad", "signature", "n_pairs")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            L.orc_cov3d_f32.argtypes = [i64, vp, vp, vp]
            L.orc_project_f32.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            L.orc_bin.argtypes = [i64, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, i64]
            L.orc_bin.restype = i64
            L.orc_sh_basis.argtypes = [ctypes.c_int, vp, vp, vp]
            L.orc_render.argtypes = [vp, vp, vp, vp, vp]
            L.orc_render_brute.argtypes = [vp, vp, vp, vp, vp]
            L.orc_se3_exp_left.argtypes = [vp, vp, vp]
            L.orc_pose_diff.argtypes = [vp, vp, vp, vp]
            _lib = L
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _cam(cam) -> _Camera:
    return _Camera(int(cam["width"]), int(cam["height"]), float(cam["fx"]), float(cam["fy"]),
                   float(cam["cx"]), float(cam["cy"]))


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(4, 4)
    return T


def cov3d_f32(scales, quats) -> np.ndarray:
    """Sec. 3.1 primitive: Sigma = R(q) diag(s)^2 R(q)^T, binary32 fixed order."""
    s = _f32(scales).reshape(-1, 3)
    q = _f32(quats).reshape(-1, 4)
    out = np.zeros((s.shape[0], 6), np.float32)
    lib().orc_cov3d_f32(s.shape[0], _p(s), _p(q), _p(out))
    return out


def project_f32(means, cov6, cam, T):
    """Algorithm 1 projection + EWA footprint + tile rectangle (binary32)."""
    m = _f32(means).reshape(-1, 3)
    c = _f32(cov6).reshape(-1, 6)
    n = m.shape[0]
    ri = np.zeros((n, 6), np.int32)
    rf = np.zeros((n, 8), np.float32)
    cc = _cam(cam)
    Tp = _pose(T)
    lib().orc_project_f32(n, _p(m), _p(c), ctypes.byref(cc), _p(Tp), _p(ri), _p(rf))
    return ri, rf


def tiles_of(cam):
    return (int(cam["width"]) + TILE - 1) // TILE, (int(cam["height"]) + TILE - 1) // TILE


def bin_tiles(rec_i, rec_f, cam):
    """Per-tile lists ordered by (binary32 depth bits, Gaussian index)."""
    tx, ty = tiles_of(cam)
    ri = np.ascontiguousarray(rec_i, np.int32)
    rf = np.ascontiguousarray(rec_f, np.float32)
    n = ri.shape[0]
    total = int(ri[ri[:, I_STATUS] == VISIBLE, I_COUNT].astype(np.int64).sum())
    ts = np.zeros(tx * ty + 1, np.int64)
    keys = np.zeros(max(total, 1), np.uint64)
    gids = np.zeros(max(total, 1), np.uint32)
    got = lib().orc_bin(n, _p(ri), _p(rf), tx, ty, _p(ts), _p(keys), _p(gids), total)
    assert got == total
    return ts, keys[:total], gids[:total]


def sh_basis(deg: int, d):
    """Real SH (Condon-Shortley) at unit direction d: values and Cartesian gradient."""
    d = np.ascontiguousarray(d, np.float64).reshape(3)
    K = (deg + 1) ** 2
    Y = np.zeros(K, np.float64)
    dY = np.zeros((K, 3), np.float64)
    lib().orc_sh_basis(deg, _p(d), _p(Y), _p(dY))
    return Y, dY


class OracleScene:
    """Holds contiguous copies of the scene arrays for the C oracle.

    unrounded_feats=True blends the scene's binary32 features ("feats_f32")
    instead of their bf16 rounding: the difference of the two renders is the
    error of bf16 feature storage alone (Sec. 3.1 features, blended like the
    colour)."""

    def __init__(self, scene: dict, unrounded_feats: bool = False):
        self.means = _f32(scene["means"]).reshape(-1, 3)
        self.n = self.means.shape[0]
        self.scales = _f32(scene["scales"]).reshape(-1, 3)
        self.quats = _f32(scene["quats"]).reshape(-1, 4)
        self.opacities = _f32(scene["opacities"]).reshape(-1)
        self.sh_degree = int(scene["sh_degree"])
        K = (self.sh_degree + 1) ** 2
        self.sh = _f32(scene["sh"]).reshape(self.n, K, 3)
        f = scene.get("feats_bf16")
        self.feats = None if f is None else np.ascontiguousarray(f, np.uint16).reshape(self.n, -1)
        self.feat_dim = 0 if self.feats is None else self.feats.shape[1]
        self.feats32 = None
        if unrounded_feats:
            self.feats32 = _f32(scene["feats_f32"]).reshape(self.n, -1)
            self.feat_dim = self.feats32.shape[1]
        self._c = _Scene(self.n, self.sh_degree, self.feat_dim, _p(self.means), _p(self.scales),
                         _p(self.quats), _p(self.opacities), _p(self.sh), _p(self.feats), _p(self.feats32))


def render(scene, cam, T, *, geom64=False, want_grad=False, n_threads=1, pixels=None,
           target_rgb=None, target_depth=None, pixel_weight=None, depth_weight=0.1,
           tie_rel=1e-4, tie_rel_T=2e-4, brute=False, want_feats=True, mean_tangent_gid=-1):
    """Full oracle render (Sec. 3.1 alpha blending; Algorithm 1 projection).

    Returns a dict of per-pixel arrays in the order of ``pixels`` (or row-major
    for the full frame): rgb (n,3), depth, alpha, final_T, last_idx, n_eval,
    n_blend, flags, feats (n,feat_dim) and, with targets, loss and grad (rho,
    phi).
    """
    sc = scene if isinstance(scene, OracleScene) else OracleScene(scene)
    W, H = int(cam["width"]), int(cam["height"])
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int64).reshape(-1)
    npx = W * H if pix is None else pix.shape[0]
    trgb = None if target_rgb is None else _f32(target_rgb).reshape(3, H, W)
    tdep = None if target_depth is None else _f32(target_depth).reshape(H, W)
    pw = None if pixel_weight is None else _f32(pixel_weight).reshape(H, W)
    opts = _Opts(int(geom64), int(want_grad), int(n_threads), _p(pix), npx, _p(trgb), _p(tdep), _p(pw),
                 float(depth_weight), float(tie_rel), float(tie_rel_T), int(mean_tangent_gid))
    res = {
        "rgb": np.zeros((npx, 3), np.float64),
        "depth": np.zeros(npx, np.float64),
        "alpha": np.zeros(npx, np.float64),
        "final_T": np.zeros(npx, np.float64),
        "last_idx": np.zeros(npx, np.int32),
        "n_eval": np.zeros(npx, np.int32),
        "n_blend": np.zeros(npx, np.int32),
        "flags": np.zeros(npx, np.uint8),
        "loss": np.zeros(1, np.float64),
        "grad": np.zeros(6, np.float64),
        "signature": np.zeros(1, np.uint64),
        "n_pairs": np.zeros(1, np.int64),
    }
    if sc.feat_dim and want_feats:
        res["feats"] = np.zeros((npx, sc.feat_dim), np.float64)
    out = _Out(*[_p(res.get(k)) for k in ("rgb", "depth", "alpha", "final_T", "last_idx", "n_eval", "n_blend",
                                           "flags", "feats", "loss", "grad", "signature", "n_pairs")])
    cc = _cam(cam)
    Tp = _pose(T)
    fn = lib().orc_render_brute if brute else lib().orc_render
    rc = fn(ctypes.byref(sc._c), ctypes.byref(cc), _p(Tp), ctypes.byref(opts), ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle render failed with code %d" % rc)
    res["loss"] = float(res["loss"][0])
    res["signature"] = int(res["signature"][0])
    res["n_pairs"] = int(res["n_pairs"][0])
    return res


def mean_gradient(scene, cam, T, gid: int, pixels=None, n_threads=1) -> dict:
    """Algorithm 1's RGB.sum().backward() for one Gaussian: the gradient of the
    sum of the rendered colours with respect to the mean of Gaussian `gid`,
    by forward differentiation in binary64 along its three mean coordinates
    (every other Gaussian held fixed). `pixels` may restrict the sum to a
    superset of the pixels the Gaussian can touch (its tile rectangle).
    Returns dict: grad (3), sum (of the colours over the pixels), flags (per
    pixel), signature."""
    r = render(scene, cam, T, geom64=True, want_grad=True, pixels=pixels, n_threads=n_threads,
               mean_tangent_gid=int(gid), want_feats=False)
    return {"grad": np.asarray(r["grad"][:3], np.float64), "sum": r["loss"], "flags": r["flags"],
            "signature": r["signature"]}


def visibility(scene, cam, T, n_threads=1, gids=None, grad_tie=1e-9, edge_tie=1e-6, want_grad=True) -> dict:
    """Algorithm 1 (render-gradient visibility check with projection filtering).

    M^r[j] = |grad_mean_j sum RGB| > 0 (mean_gradient over the pixels of the
    tiles Gaussian j covers), M^i[j] = the projection (u, v) = K (p / z) lies in
    [0, W) x [0, H), M = M^i and M^r. Evaluated for every Gaussian, or for
    `gids`. Returns dict over those Gaussians: gids, grad (n, 3), M_r, M_i, M,
    uv (n, 2), flag (a decision within rounding: a gradient below grad_tie
    relative to the largest, a zero gradient with a near-tie pixel in its
    rectangle, or (u, v) within edge_tie of an image edge). want_grad=False
    evaluates the projection part only (grad, M_r and M are then all zero)."""
    cov = cov3d_f32(scene["scales"], scene["quats"])
    ri, rf = project_f32(scene["means"], cov, cam, T)
    W, H = int(cam["width"]), int(cam["height"])
    n = ri.shape[0]
    gids = np.arange(n) if gids is None else np.asarray(gids, np.int64)
    Tm = np.asarray(T, np.float64)
    p = np.asarray(scene["means"], np.float64)[gids] @ Tm[:3, :3].T + Tm[:3, 3]
    fx, fy, cx, cy = (float(np.float32(cam[k])) for k in ("fx", "fy", "cx", "cy"))
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * p[:, 0] / p[:, 2] + cx
        v = fy * p[:, 1] / p[:, 2] + cy
    M_i = (u >= 0) & (u < W) & (v >= 0) & (v < H)
    grad = np.zeros((len(gids), 3))
    tie_px = np.zeros(len(gids), bool)
    for k, g in enumerate(gids):
        if not want_grad or ri[g, I_STATUS] != VISIBLE:
            continue
        x0, x1, y0, y1 = (int(ri[g, c]) for c in (I_X0, I_X1, I_Y0, I_Y1))
        ys, xs = np.mgrid[y0 * TILE:min(H, (y1 + 1) * TILE), x0 * TILE:min(W, (x1 + 1) * TILE)]
        pix = (ys * W + xs).reshape(-1).astype(np.int64)
        r = mean_gradient(scene, cam, T, int(g), pixels=pix, n_threads=n_threads)
        grad[k] = r["grad"]
        tie_px[k] = bool((r["flags"] & TIE_IMAGE).any())
    norm = np.linalg.norm(grad, axis=1)
    M_r = norm > 0
    big = norm.max() if len(norm) else 0.0
    edge = (np.abs(u) <= edge_tie * W) | (np.abs(u - W) <= edge_tie * W) | (np.abs(v) <= edge_tie * H) | \
        (np.abs(v - H) <= edge_tie * H)
    flag = ((norm > 0) & (norm <= grad_tie * big)) | ((norm == 0) & tie_px) | edge
    return {"gids": gids, "grad": grad, "M_r": M_r, "M_i": M_i, "M": M_r & M_i,
            "uv": np.stack([u, v], 1), "flag": flag}


def se3_exp_left(xi, T) -> np.ndarray:
    """Left update T' = Exp(xi^) T with xi = (rho, phi)."""
    x = np.ascontiguousarray(xi, np.float64).reshape(6)
    Tp = _pose(T)
    out = np.zeros((4, 4), np.float64)
    lib().orc_se3_exp_left(_p(x), _p(Tp), _p(out))
    return out


def pose_diff(T1, T2):
    """Algorithm 2: angle (deg) of R1 R2^T with the trace clamp, and |t1 - t2|."""
    a = np.zeros(1, np.float64)
    d = np.zeros(1, np.float64)
    P1, P2 = _pose(T1), _pose(T2)
    lib().orc_pose_diff(_p(P1), _p(P2), _p(a), _p(d))
    return float(a[0]), float(d[0])
