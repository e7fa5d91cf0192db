"""Probabilistic mutual matching (PMM) of Sec. 3.4, Eq. 11 -- fp64 oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg of
``bench.py``, never by the product path.

Sec. 3.4 matches a query feature map against the feature map rendered at the
current pose, coarse to fine: at the coarse level (H_f / H_c = 8) the cosine
similarity matrix M of all coarse positions, the dual softmax
    P_M = softmax_j(M / tau) * softmax_i(M / tau)                    (Eq. 11)
and mutual nearest neighbours (MNN) on P_M give the coarse correspondences;
inside the w x w windows (w = H_f / H_c) at each coarse correspondence the same
operations on the fine features give the fine correspondences.

Readings where the paper is silent (the same in the CUDA path):
* coarse maps are the 8 x 8 block means of the fine maps (H, W multiples of 8);
* feature vectors are L2-normalised before the dot product (cosine); a zero
  vector stays zero (similarity 0 with everything);
* the definition has no rounding of its own: the coarse level here is binary64
  throughout (block means of the binary32 fine map, their norms and the
  cosine matrix), i.e. Eq. 11 on the unrounded cell means;
* tau = 0.1;
* MNN: i and j match when j is the first index of the maximum of row i of P_M
  and i the first index of the maximum of column j;
* fine level: the window of a coarse position is its 8 x 8 block of fine
  pixels; fine vectors are normalised in binary64; the dual softmax and MNN run
  on the 64 x 64 similarity of the two windows; the fine correspondence is
  reported as fine pixel indices.

Decisions taken within rounding of a tie (the best and second-best log P_M of a
row or column closer than ``TIE_GAP``) are flagged; parity tests compare the
unflagged decisions exactly.

A second, documented precision layer (``coarse_codes_bf16``,
``coarse_pmm_bf16``) rounds the coarse unit vectors to bfloat16, as a plain
single-bf16 tensor-core contraction would: it is not the definition, and it
exists to measure how many coarse decisions and matches such a contraction
changes against the definition (``decision_changes``).
"""
from __future__ import annotations

import numpy as np

RATIO = 8
TAU = 0.1
TIE_GAP = 1e-3  # in log P units: fp32 similarities and log-sum-exps on the GPU err by ~1e-4 at most


def _bf16_round_bits(x32: np.ndarray) -> np.ndarray:
    """Round binary32 to bfloat16, nearest even (finite inputs), as bit patterns."""
    u = np.ascontiguousarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def coarse_unit_means(F: np.ndarray, ratio: int = RATIO) -> np.ndarray:
    """The coarse unit feature vectors of the definition, (Hc * Wc, C) fp64.

    F: (C, H, W) fine feature map (binary32 values, widened exactly). Cell
    (cy, cx) is the mean of its ratio x ratio block, divided by its Euclidean
    norm; a zero mean stays zero."""
    F = np.asarray(F, np.float32)
    C, H, W = F.shape
    assert H % ratio == 0 and W % ratio == 0, "feature maps must be multiples of the coarse ratio"
    Hc, Wc = H // ratio, W // ratio
    m = F.astype(np.float64).reshape(C, Hc, ratio, Wc, ratio).mean(axis=(2, 4)).reshape(C, Hc * Wc).T
    n = np.linalg.norm(m, axis=1, keepdims=True)
    return np.where(n > 0, m / np.where(n > 0, n, 1.0), 0.0)


def coarse_codes_bf16(F: np.ndarray, ratio: int = RATIO) -> np.ndarray:
    """Precision layer, not the definition: coarse unit feature vectors rounded
    to bfloat16 bits, (Hc * Wc, C) row-major, as a single-bf16 contraction
    would take them.

    F: (C, H, W) fine feature map (binary32). Block mean: s = sum over the block
    in row-major order, then s * (1 / ratio^2) (exact); norm: sequential sum of
    m_c * m_c over channels, sqrt, one division per channel; all binary32."""
    F = np.ascontiguousarray(F, np.float32)
    C, H, W = F.shape
    assert H % ratio == 0 and W % ratio == 0, "feature maps must be multiples of the coarse ratio"
    Hc, Wc = H // ratio, W // ratio
    blk = F.reshape(C, Hc, ratio, Wc, ratio)
    s = np.zeros((C, Hc, Wc), np.float32)
    for dy in range(ratio):
        for dx in range(ratio):
            s = (s + blk[:, :, dy, :, dx]).astype(np.float32)
    m = (s * np.float32(1.0 / (ratio * ratio))).astype(np.float32)
    ss = np.zeros((Hc, Wc), np.float32)
    for c in range(C):
        ss = (ss + (m[c] * m[c]).astype(np.float32)).astype(np.float32)
    n = np.sqrt(ss).astype(np.float32)
    safe = np.where(n > 0, n, np.float32(1.0)).astype(np.float32)
    u = np.where(n > 0, (m / safe).astype(np.float32), np.float32(0.0)).astype(np.float32)
    return _bf16_round_bits(u.reshape(C, Hc * Wc).T.copy())


def log_dual_softmax(M: np.ndarray, tau: float = TAU):
    """Eq. 11 in log form: log P_M = 2 M / tau - r_i - c_j with r, c the row and
    column log-sum-exps of M / tau. Returns (logP, r, c)."""
    A = np.asarray(M, np.float64) / tau
    rmax = A.max(axis=1, keepdims=True)
    r = (rmax + np.log(np.exp(A - rmax).sum(axis=1, keepdims=True)))[:, 0]
    cmax = A.max(axis=0, keepdims=True)
    c = (cmax + np.log(np.exp(A - cmax).sum(axis=0, keepdims=True)))[0]
    return 2.0 * A - r[:, None] - c[None, :], r, c


def _best_and_gap(L: np.ndarray, axis: int):
    """First index of the maximum along `axis` and the gap to the runner-up."""
    best = np.argmax(L, axis=axis)
    top = np.take_along_axis(L, np.expand_dims(best, axis), axis).squeeze(axis)
    if L.shape[axis] < 2:
        return best, np.full(best.shape, np.inf)
    part = -np.partition(-L, 1, axis=axis)
    second = np.take(part, 1, axis=axis)
    return best, top - second


def mnn(logP: np.ndarray, tie_gap: float = TIE_GAP):
    """Mutual nearest neighbours on P_M (maxima of log P_M, first index on ties).

    Returns dict: row_best (Nq), col_best (Nr), row_gap, col_gap, matches
    (K, 2) int64 sorted by query index, prob (K), row_flag / col_flag (gap below
    tie_gap)."""
    rb, rgap = _best_and_gap(logP, 1)
    cb, cgap = _best_and_gap(logP, 0)
    i = np.arange(logP.shape[0])
    mutual = cb[rb] == i
    mi = i[mutual]
    mj = rb[mutual]
    return {"row_best": rb, "col_best": cb, "row_gap": rgap, "col_gap": cgap,
            "row_flag": rgap < tie_gap, "col_flag": cgap < tie_gap,
            "matches": np.stack([mi, mj], 1).astype(np.int64), "prob": np.exp(logP[mi, mj])}


def coarse_pmm(Fq: np.ndarray, Fr: np.ndarray, tau: float = TAU, ratio: int = RATIO) -> dict:
    """Coarse level of Sec. 3.4 (the definition): fp64 unit cell means, their
    cosine matrix M, Eq. 11, MNN. Returns mnn()'s dict plus the unit means
    ("units_q", "units_r"), the row / column log-sum-exps and M."""
    uq = coarse_unit_means(Fq, ratio)
    ur = coarse_unit_means(Fr, ratio)
    M = uq @ ur.T
    logP, r, c = log_dual_softmax(M, tau)
    out = mnn(logP)
    out.update({"units_q": uq, "units_r": ur, "lse_row": r, "lse_col": c, "M": M})
    return out


def coarse_pmm_bf16(Fq: np.ndarray, Fr: np.ndarray, tau: float = TAU, ratio: int = RATIO) -> dict:
    """Precision layer, not the definition: the coarse level on bf16-rounded
    unit means (exact fp64 products of the rounded vectors)."""
    cq = coarse_codes_bf16(Fq, ratio)
    cr = coarse_codes_bf16(Fr, ratio)
    M = bf16_to_f64(cq) @ bf16_to_f64(cr).T
    logP, r, c = log_dual_softmax(M, tau)
    out = mnn(logP)
    out.update({"codes_q": cq, "codes_r": cr, "lse_row": r, "lse_col": c, "M": M})
    return out


def decision_changes(a: dict, ref: dict) -> dict:
    """How many coarse decisions and matches of `a` differ from those of `ref`
    (two outputs of coarse_pmm-like functions on the same maps): fractions of
    row argmaxes, column argmaxes and of the union of the match sets, overall
    and among the decisions that `ref` takes clear of a tie."""
    rd = a["row_best"] != ref["row_best"]
    cd = a["col_best"] != ref["col_best"]
    ma = {tuple(x) for x in np.asarray(a["matches"]).tolist()}
    mr = {tuple(x) for x in np.asarray(ref["matches"]).tolist()}
    rok, cok = ~ref["row_flag"], ~ref["col_flag"]
    clear = lambda ij: rok[ij[0]] and cok[ij[1]]
    ca, cr = {x for x in ma if clear(x)}, {x for x in mr if clear(x)}
    return {"row": float(rd.mean()), "col": float(cd.mean()),
            "row_clear": float(rd[rok].mean()) if rok.any() else 0.0,
            "col_clear": float(cd[cok].mean()) if cok.any() else 0.0,
            "matches": len(ma ^ mr) / max(1, len(ma | mr)),
            "matches_clear": len(ca ^ cr) / max(1, len(ca | cr)),
            "row_flagged": float(ref["row_flag"].mean()), "col_flagged": float(ref["col_flag"].mean())}


def _window(F: np.ndarray, cell: int, Wc: int, ratio: int) -> np.ndarray:
    y0, x0 = (cell // Wc) * ratio, (cell % Wc) * ratio
    v = np.asarray(F[:, y0:y0 + ratio, x0:x0 + ratio], np.float64).reshape(F.shape[0], -1).T
    n = np.linalg.norm(v, axis=1, keepdims=True)
    return np.where(n > 0, v / np.where(n > 0, n, 1.0), 0.0)


def fine_pmm(Fq: np.ndarray, Fr: np.ndarray, coarse_matches: np.ndarray, tau: float = TAU,
             ratio: int = RATIO) -> dict:
    """Fine level of Sec. 3.4: for each coarse match (i, j) the 64 x 64 cosine
    matrix of the w x w windows (w = ratio) of fine pixels of cell i (query) and
    cell j (rendered), Eq. 11 and MNN inside the window pair.

    Returns dict: matches (K, 3) int64 rows (coarse match index, query fine
    pixel, rendered fine pixel) with pixels as y * W + x, prob (K), flag (K)
    (a near-tie decision on that row or column)."""
    C, H, W = Fq.shape
    Wc = W // ratio
    rows, probs, flags = [], [], []
    for k, (i, j) in enumerate(np.asarray(coarse_matches, np.int64)):
        uq = _window(Fq, int(i), Wc, ratio)
        ur = _window(Fr, int(j), Wc, ratio)
        logP, _, _ = log_dual_softmax(uq @ ur.T, tau)
        m = mnn(logP)
        for a, b in m["matches"]:
            qy, qx = (i // Wc) * ratio + a // ratio, (i % Wc) * ratio + a % ratio
            ry, rx = (j // Wc) * ratio + b // ratio, (j % Wc) * ratio + b % ratio
            rows.append((k, qy * W + qx, ry * W + rx))
            probs.append(np.exp(logP[a, b]))
            flags.append(bool(m["row_flag"][a] or m["col_flag"][b]))
    return {"matches": np.asarray(rows, np.int64).reshape(-1, 3), "prob": np.asarray(probs, np.float64),
            "flag": np.asarray(flags, bool)}


def coarse_pmm_chunked(Fq: np.ndarray, Fr: np.ndarray, tau: float = TAU, ratio: int = RATIO,
                       chunk: int = 2048, tie_gap: float = TIE_GAP, bf16: bool = False) -> dict:
    """coarse_pmm (or, with bf16=True, the precision layer coarse_pmm_bf16) for
    maps whose full similarity matrix does not fit in memory: the same
    formulas over blocks of query rows (M is never stored whole). Returns the
    same keys except "M"."""
    if bf16:
        cq, cr = coarse_codes_bf16(Fq, ratio), coarse_codes_bf16(Fr, ratio)
        Q, R = bf16_to_f64(cq), bf16_to_f64(cr)
        extra = {"codes_q": cq, "codes_r": cr}
    else:
        Q, R = coarse_unit_means(Fq, ratio), coarse_unit_means(Fr, ratio)
        extra = {"units_q": Q, "units_r": R}
    n_q, n_r = Q.shape[0], R.shape[0]
    # pass 1: row log-sum-exps; column log-sum-exps from per-block maxima and sums
    r = np.empty(n_q)
    cmax = np.full(n_r, -np.inf)
    for s in range(0, n_q, chunk):
        A = (Q[s:s + chunk] @ R.T) / tau
        m = A.max(axis=1, keepdims=True)
        r[s:s + chunk] = (m + np.log(np.exp(A - m).sum(axis=1, keepdims=True)))[:, 0]
        cmax = np.maximum(cmax, A.max(axis=0))
    csum = np.zeros(n_r)
    for s in range(0, n_q, chunk):
        A = (Q[s:s + chunk] @ R.T) / tau
        csum += np.exp(A - cmax[None, :]).sum(axis=0)
    c = cmax + np.log(csum)
    # pass 2: best and runner-up of rows and columns of log P_M
    rb = np.empty(n_q, np.int64)
    rgap = np.empty(n_q)
    ctop = np.full(n_r, -np.inf)
    csec = np.full(n_r, -np.inf)
    cb = np.zeros(n_r, np.int64)
    for s in range(0, n_q, chunk):
        L = 2.0 * (Q[s:s + chunk] @ R.T) / tau - r[s:s + chunk, None] - c[None, :]
        b, gap = _best_and_gap(L, 1)
        rb[s:s + chunk], rgap[s:s + chunk] = b, gap
        # columns: merge this block's top two into the running top two (first index kept on ties)
        bi = np.argmax(L, axis=0)
        bt = L[bi, np.arange(n_r)]
        L2 = L.copy()
        L2[bi, np.arange(n_r)] = -np.inf
        bs = L2.max(axis=0) if L.shape[0] > 1 else np.full(n_r, -np.inf)
        new_top = bt > ctop
        csec = np.where(new_top, np.maximum(ctop, bs), np.maximum(csec, bt))
        cb = np.where(new_top, s + bi, cb)
        ctop = np.where(new_top, bt, ctop)
    cgap = ctop - csec
    i = np.arange(n_q)
    mutual = cb[rb] == i
    mi, mj = i[mutual], rb[mutual]
    prob = np.exp(2.0 * np.einsum("ij,ij->i", Q[mi], R[mj]) / tau - r[mi] - c[mj])
    out = {"row_best": rb, "col_best": cb, "row_gap": rgap, "col_gap": cgap, "row_flag": rgap < tie_gap,
           "col_flag": cgap < tie_gap, "matches": np.stack([mi, mj], 1).astype(np.int64), "prob": prob,
           "lse_row": r, "lse_col": c}
    out.update(extra)
    return out
