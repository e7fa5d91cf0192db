"""Helpers shared by the GPU parity tests (comparison only; no method arithmetic)."""
import numpy as np

# Max-abs tolerance of an fp32 image against the fp64 oracle, relative to the
# output's own scale max(1, max|oracle|): 1e-4 (rgb, alpha, transmittance are
# O(1); depth is compared relative to the largest depth).
IMAGE_TOL = 1e-4
GRAD_TOL = 1e-3


def to_numpy(out, H, W):
    r = {k: v.detach().cpu().numpy() for k, v in out.items()}
    res = {"rgb": r["rgb"].reshape(3, H * W).T.astype(np.float64),
           "depth": r["depth"].reshape(-1).astype(np.float64),
           "alpha": r["alpha"].reshape(-1).astype(np.float64),
           "final_T": r["final_T"].reshape(-1).astype(np.float64)}
    if "last_idx" in r:
        res["last_idx"] = r["last_idx"].reshape(-1).astype(np.int64)
    if "feats" in r:
        res["feats"] = r["feats"].reshape(r["feats"].shape[0], H * W).T.astype(np.float64)
    return res


def compare_images(gpu, orc, oracle_mod, pixels=None, tol=IMAGE_TOL, min_ok=0.99):
    """Compare on pixels without a near-tie decision; check the rest is valid.
    Returns the max scaled errors per output."""
    sel = slice(None) if pixels is None else pixels
    ok = (orc["flags"] & oracle_mod.TIE_IMAGE) == 0
    assert ok.mean() >= min_ok, "too many near-tie pixels: %.4f" % ok.mean()
    errs = {}
    for k in ("rgb", "depth", "alpha", "final_T", "feats"):
        if k not in orc or k not in gpu:
            continue
        g = gpu[k][sel]
        o = orc[k]
        scale = max(1.0, float(np.abs(o).max()) if o.size else 1.0)
        d = np.abs(g - o)
        if d.ndim > 1:
            d = d.max(axis=1)
        errs[k] = float(d[ok].max() / scale) if ok.any() else 0.0
        assert errs[k] <= tol, "%s: max scaled error %.3g > %.1g" % (k, errs[k], tol)
        assert np.all(np.isfinite(g)), k
    if "last_idx" in gpu:
        np.testing.assert_array_equal(gpu["last_idx"][sel][ok], orc["last_idx"][ok])
    # near-tie pixels: valid values only
    a = gpu["alpha"][sel]
    assert np.all((a >= 0) & (a < 1))
    assert np.all(gpu["final_T"][sel] >= 1e-4 * (1 - 1e-5))
    assert np.all(gpu["rgb"][sel] >= 0)
    return errs


def block_rel_err(g, ref):
    """Relative error of the translation and rotation blocks of a 6-vector gradient."""
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    out = []
    for s in (slice(0, 3), slice(3, 6)):
        out.append(float(np.linalg.norm(g[s] - ref[s]) / max(np.linalg.norm(ref[s]), 1e-30)))
    return out


def component_rel_err(g, ref):
    """Relative error of each of the six gradient components, |g_k - ref_k| / |ref_k|."""
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    return [float(abs(g[k] - ref[k]) / max(abs(ref[k]), 1e-300)) for k in range(6)]
