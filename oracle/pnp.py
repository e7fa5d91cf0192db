"""Dense PnP + RANSAC on rendered depth (Sec. 3.4, Eq. 10) -- fp64 oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg of
``bench.py``, never by the product path.

Sec. 3.4 closes each coarse-to-fine round with a 2D-3D PnP solved by RANSAC:
the 3D point of a dense match is its rendered pixel lifted through the
rendered depth at the render pose; Eq. 10 chooses the pose and inlier set that
minimise a robust reprojection loss rho(||p - pi(K [R|t] g)||, tau).

Readings where the paper is silent (the same in the CUDA path):
* one pinhole camera K for the query and the rendered maps (the maps are
  matched pixel to pixel, so they share the size); pixel (x, y) has centre
  (x + 0.5, y + 0.5);
* lifting: the rendered depth is the un-normalised sum of w z, so the depth of
  the surface seen at a pixel is D / alpha; pixels with alpha < min_alpha
  (0.5) give no 3D point; the lifted point is R_r^T (z K^-1 (x+.5, y+.5, 1) - t_r);
* the robust loss is the truncated square rho(e) = min(e, tau)^2: RANSAC
  keeps the minimal-sample pose with the most inliers (e < tau, point in front
  of the camera), ties to the lowest hypothesis and solution index; the pose
  is then refined by Gauss-Newton on the sum of squared errors of the current
  inliers (re-selected before every step), left se(3) updates xi = (rho, phi);
* minimal solver: P3P after Grunert (as reviewed by Haralick et al., 1994):
  with u = s2 / s1 and v = s3 / s1 the law of cosines gives
  u = N(v) / (2 D(v)) and a quartic Q(v) = 4 D^2 E + N^2 - 4 cos(gamma) N D
  (polynomials below), formed here by polynomial products; every real root
  with v > 0, D(v) != 0, u > 0 gives the three distances, and the pose comes
  from the two point triads (orthonormal frames of both triangles).
  Solutions are ordered by ascending v;
* random numbers: hypothesis h draws three uint32 words w (inputs); its match
  indices are floor(w K / 2^32) over the K matches with depth (in match
  order); a sample with a repeated index or a degenerate triangle has no
  solution.

Near-threshold decisions (|e - tau| < TIE_PX) and quartics with a near-double
root are flagged; parity tests compare what is clear of them.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as _orc

TIE_PX = 1e-3       # reprojection errors this close to tau are decided within rounding
MIN_ALPHA = 0.5


def _cam(cam):
    return float(np.float32(cam["fx"])), float(np.float32(cam["fy"])), float(np.float32(cam["cx"])), \
        float(np.float32(cam["cy"]))


def lift(depth, alpha, cam, T_r, matches, min_alpha=MIN_ALPHA):
    """3D world point of each match's rendered pixel and its query pixel centre.

    depth, alpha: (H, W) renders at pose T_r (world-to-camera 4x4); matches:
    (K, 3) rows (coarse index, query pixel, rendered pixel), pixels y W + x.
    Returns X (K, 3), p (K, 2), valid (K) bool."""
    W = int(cam["width"])
    fx, fy, cx, cy = _cam(cam)
    m = np.asarray(matches, np.int64).reshape(-1, 3)
    q, r = m[:, 1], m[:, 2]
    D = np.asarray(depth, np.float64).reshape(-1)[r]
    A = np.asarray(alpha, np.float64).reshape(-1)[r]
    valid = A >= min_alpha
    z = np.where(valid, D / np.where(valid, A, 1.0), 0.0)
    xc = np.stack([z * ((r % W) + 0.5 - cx) / fx, z * ((r // W) + 0.5 - cy) / fy, z], 1)
    T = np.asarray(T_r, np.float64)
    X = (xc - T[:3, 3]) @ T[:3, :3]  # R^T (xc - t)
    p = np.stack([(q % W) + 0.5, (q // W) + 0.5], 1).astype(np.float64)
    return X, p, valid


def bearings(p, cam):
    fx, fy, cx, cy = _cam(cam)
    f = np.stack([(p[:, 0] - cx) / fx, (p[:, 1] - cy) / fy, np.ones(len(p))], 1)
    return f / np.linalg.norm(f, axis=1, keepdims=True)


def _frame(P):
    e1 = P[1] - P[0]
    n = np.cross(e1, P[2] - P[0])
    e1 = e1 / np.linalg.norm(e1)
    n = n / np.linalg.norm(n)
    return np.stack([e1, np.cross(n, e1), n], 1)  # columns


def triad_pose(X, Q):
    """(R, t) with Q_i = R X_i + t for two congruent triangles (3 x 3 rows)."""
    R = _frame(Q) @ _frame(X).T
    return R, Q[0] - R @ X[0]


def quartic(X, f):
    """Grunert's quartic in v for world points X (3 x 3) and unit bearings f.
    Returns (coefficients low -> high, helpers) or None for a degenerate sample."""
    a2 = float(np.sum((X[1] - X[2]) ** 2))
    b2 = float(np.sum((X[0] - X[2]) ** 2))
    c2 = float(np.sum((X[0] - X[1]) ** 2))
    if b2 <= 0.0 or a2 <= 0.0 or c2 <= 0.0:
        return None
    ca, cb, cg = float(f[1] @ f[2]), float(f[0] @ f[2]), float(f[0] @ f[1])
    k = (a2 - c2) / b2
    P = np.polynomial.polynomial
    D = np.array([cg, -ca])
    N = np.array([1.0 + k, -2.0 * k * cb, k - 1.0])
    E = np.array([1.0 - c2 / b2, 2.0 * (c2 / b2) * cb, -c2 / b2])
    Q = P.polyadd(P.polyadd(4.0 * P.polymul(P.polymul(D, D), E), P.polymul(N, N)), -4.0 * cg * P.polymul(N, D))
    Q = np.concatenate([Q, np.zeros(5 - len(Q))])
    return Q, (a2, b2, c2, ca, cb, cg, D, N)


def real_roots(Q):
    """Real roots of the quartic (coefficients low -> high), polished by Newton.
    Also returns whether the quartic has a near-double real root."""
    P = np.polynomial.polynomial
    if Q[4] == 0.0:
        return np.zeros(0), True
    z = np.roots(Q[::-1])
    scale = np.maximum(1.0, np.abs(z))
    re = np.sort(z[np.abs(z.imag) <= 1e-7 * scale].real)
    dQ = P.polyder(Q)
    out = []
    for x in re:
        for _ in range(4):
            d = P.polyval(x, dQ)
            if d == 0.0:
                break
            x = x - P.polyval(x, Q) / d
        out.append(x)
    out = np.asarray(out)
    # near-double root: two of the four (complex) roots closer than 1e-4 of their scale
    gap = np.where(np.eye(len(z), dtype=bool), np.inf, np.abs(z[:, None] - z[None, :]))
    near = bool(np.any(gap < 1e-4 * np.maximum(scale[:, None], scale[None, :])))
    return out, near


def p3p(X, f):
    """All P3P poses (R, t) for 3 world points and unit bearings, by ascending v.
    Returns (list of (R, t, v), near_double_root)."""
    qq = quartic(X, f)
    if qq is None:
        return [], False
    Q, (a2, b2, c2, ca, cb, cg, D, N) = qq
    if np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0])) <= 1e-12 * (a2 + b2 + c2):
        return [], False
    P = np.polynomial.polynomial
    roots, near = real_roots(Q)
    sols = []
    for v in roots:
        if not v > 0.0:
            continue
        Dv = P.polyval(v, D)
        if Dv == 0.0:
            continue
        u = P.polyval(v, N) / (2.0 * Dv)
        if not u > 0.0:
            continue
        s1 = np.sqrt(b2 / (1.0 + v * v - 2.0 * v * cb))
        Qc = np.stack([s1 * f[0], u * s1 * f[1], v * s1 * f[2]])
        R, t = triad_pose(X, Qc)
        sols.append((R, t, float(v)))
    return sols, near


def sample_indices(words, K):
    """Match indices of each hypothesis: floor(w K / 2^32)."""
    w = np.asarray(words, np.uint64).reshape(-1, 3)
    return ((w * np.uint64(K)) >> np.uint64(32)).astype(np.int64)


def reproj_err(R, t, X, p, cam):
    fx, fy, cx, cy = _cam(cam)
    pc = X @ np.asarray(R).T + np.asarray(t)
    z = pc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * pc[:, 0] / z + cx
        v = fy * pc[:, 1] / z + cy
    e = np.hypot(u - p[:, 0], v - p[:, 1])
    return np.where(z > 0, e, np.inf), pc


def inliers(R, t, X, p, cam, tau):
    """(inlier mask, near-threshold mask) under pose (R, t)."""
    e, _ = reproj_err(R, t, X, p, cam)
    return e < tau, np.abs(e - tau) < TIE_PX


def ransac(X, p, cam, words, tau):
    """RANSAC over P3P hypotheses on the matches with depth (X, p: K rows).

    Returns dict: hyps (list per hypothesis of solutions (R, t, v)), counts
    (list of per-solution inlier counts), ambiguous (per-solution counts of
    near-threshold matches), near_root (per hypothesis), best (h, s) or None,
    best_count."""
    K = len(X)
    idx = sample_indices(words, K)
    f = bearings(p, cam)
    hyps, counts, amb, nears = [], [], [], []
    best, best_c = None, -1
    for h, (i, j, k) in enumerate(idx):
        if K < 3 or i == j or i == k or j == k:
            hyps.append([]); counts.append([]); amb.append([]); nears.append(False)
            continue
        sel = np.array([i, j, k])
        sols, near = p3p(X[sel], f[sel])
        hyps.append(sols)
        nears.append(near)
        cs, am = [], []
        for s, (R, t, _) in enumerate(sols):
            inl, tie = inliers(R, t, X, p, cam, tau)
            c = int(inl.sum())
            cs.append(c)
            am.append(int(tie.sum()))
            if c > best_c:
                best, best_c = (h, s), c
        counts.append(cs)
        amb.append(am)
    return {"idx": idx, "hyps": hyps, "counts": counts, "ambiguous": amb, "near_root": nears, "best": best,
            "best_count": best_c}


def gn_refine(T, X, p, cam, tau, iters):
    """Gauss-Newton on the squared reprojection errors of the inliers, which are
    re-selected under the current pose before each step; left updates
    T <- Exp(xi) T with xi = -(J^T J)^-1 J^T e. Returns (T, history of inlier counts)."""
    fx, fy, _, _ = _cam(cam)
    T = np.asarray(T, np.float64).copy()
    hist = []
    for _ in range(iters):
        R, t = T[:3, :3], T[:3, 3]
        inl, _ = inliers(R, t, X, p, cam, tau)
        hist.append(int(inl.sum()))
        if inl.sum() < 3:
            break
        e_all, pc = reproj_err(R, t, X, p, cam)
        pc = pc[inl]
        x, y, z = pc[:, 0], pc[:, 1], pc[:, 2]
        u = fx * x / z + _cam(cam)[2]
        v = fy * y / z + _cam(cam)[3]
        r = np.stack([u - p[inl, 0], v - p[inl, 1]], 1)  # residual (n, 2)
        dpi = np.zeros((len(pc), 2, 3))
        dpi[:, 0, 0] = fx / z
        dpi[:, 0, 2] = -fx * x / (z * z)
        dpi[:, 1, 1] = fy / z
        dpi[:, 1, 2] = -fy * y / (z * z)
        dp = np.zeros((len(pc), 3, 6))
        dp[:, :, :3] = np.eye(3)
        # d p / d phi = -[p]x
        dp[:, 0, 4], dp[:, 0, 5] = z, -y
        dp[:, 1, 3], dp[:, 1, 5] = -z, x
        dp[:, 2, 3], dp[:, 2, 4] = y, -x
        J = np.einsum("nij,njk->nik", dpi, dp)  # (n, 2, 6)
        H = np.einsum("nij,nik->jk", J, J)
        g = np.einsum("nij,ni->j", J, r)
        try:
            xi = -np.linalg.solve(H, g)
        except np.linalg.LinAlgError:
            break
        T = _orc.se3_exp_left(xi, T)
    return T, hist


def pnp_ransac(depth, alpha, cam, T_r, matches, words, tau=2.0, refine_iters=10, min_alpha=MIN_ALPHA):
    """Eq. 10 on dense matches: lift, RANSAC over P3P hypotheses, Gauss-Newton
    refinement on the inliers. Returns dict with pose T (4x4), n_inliers,
    inlier (K_valid mask over the matches with depth), valid (over all
    matches), the RANSAC record and the refinement history."""
    X, p, valid = lift(depth, alpha, cam, T_r, matches, min_alpha)
    Xv, pv = X[valid], p[valid]
    rs = ransac(Xv, pv, cam, words, tau)
    out = {"X": Xv, "p": pv, "valid": valid, "ransac": rs}
    if rs["best"] is None:
        out.update({"T": np.asarray(T_r, np.float64).copy(), "n_inliers": 0,
                    "inlier": np.zeros(len(Xv), bool), "history": []})
        return out
    h, s = rs["best"]
    R, t, _ = rs["hyps"][h][s]
    T0 = np.eye(4)
    T0[:3, :3], T0[:3, 3] = R, t
    T, hist = gn_refine(T0, Xv, pv, cam, tau, refine_iters)
    inl, tie = inliers(T[:3, :3], T[:3, 3], Xv, pv, cam, tau)
    out.update({"T": T, "T_best": T0, "n_inliers": int(inl.sum()), "inlier": inl, "tie": tie, "history": hist})
    return out
