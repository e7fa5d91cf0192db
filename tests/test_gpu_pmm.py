"""GPU probabilistic mutual matching (Sec. 3.4, Eq. 11) against the oracle,
through the C ABI (gs_pmm_*).

Inputs are feature maps rendered by the oracle (32 channels, fp32) at a
reference and a perturbed pose. The oracle's coarse level is the definition
(fp64 unit cell means, no rounding of its own). The library's split codes
(hi + lo bfloat16) must equal the fp64 unit means to 2e-5; the row / column
log-sum-exps agree to 1e-5; every argmax decision and coarse or fine match
whose margin is not within rounding of a tie (oracle flag) must be identical,
and at least the stated fraction of decisions must be clear of ties. Each
test also prints how many coarse decisions and matches a plain single-bf16
contraction (the oracle's precision layer) would change.
"""
import math

import numpy as np
import pytest
import torch

from oracle import pmm as OP
from paper_2507_15683_gb300 import synth

pytestmark = pytest.mark.gpu

# Fractions of the coarse decisions clear of ties under the definition, as the
# oracle measures them on these maps, less a margin: 510 cells 1.0 / 1.0 (rows
# / columns), 4160 cells 0.9986 / 0.9978, 1080p 0.99966 / 0.99948.
MIN_CLEAR_SMALL = 0.995
MIN_CLEAR_1080P = 0.999


def _maps(oracle, seed, w, h, f, n=20000, angle=2.0, move=2.0):
    scene = synth.aerial_scene(seed, n, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20, feat_dim=32)
    cam = synth.camera(w, h, f)
    T = synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0))
    Tq = synth.perturb_pose(T, synth.rng(seed + 1), angle, move)
    out = []
    for pose in (T, Tq):
        r = oracle.render(scene, cam, pose, geom64=True, n_threads=16)
        out.append(np.ascontiguousarray(r["feats"].T.reshape(32, h, w).astype(np.float32)))
    return out


def _gpu(gsr, Fq, Fr, tau=OP.TAU):
    m = gsr.Matcher(Fq.shape[1], Fq.shape[2])
    res = m.match(torch.from_numpy(Fq).cuda(), torch.from_numpy(Fr).cuda(), tau)
    m.close()
    return {k: v.cpu().numpy() for k, v in res.items()}


def _split_units(codes):
    """(n, 64) bf16 hi[32], lo[32] -> hi + lo in fp64, after checking that lo is
    below half a bf16 unit of hi (hi is the rounded value)."""
    hi, lo = OP.bf16_to_f64(codes[:, :32]), OP.bf16_to_f64(codes[:, 32:])
    assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -8 + 1e-30)
    return hi + lo


def _check_coarse(g, o, min_clear, label, Fq=None, Fr=None):
    np.testing.assert_allclose(_split_units(g["codes_q"]), o["units_q"], rtol=0, atol=2e-5)
    np.testing.assert_allclose(_split_units(g["codes_r"]), o["units_r"], rtol=0, atol=2e-5)
    np.testing.assert_allclose(g["lse_row"], o["lse_row"], rtol=1e-5)
    np.testing.assert_allclose(g["lse_col"], o["lse_col"], rtol=1e-5)
    rok, cok = ~o["row_flag"], ~o["col_flag"]
    print("\n%s: clear of ties: rows %.5f, columns %.5f (floor %.3f)" % (label, rok.mean(), cok.mean(), min_clear))
    if Fq is not None:  # what a single-bf16 contraction would change against the definition
        b = (OP.coarse_pmm_chunked(Fq, Fr, bf16=True) if len(rok) > 8192 else OP.coarse_pmm_bf16(Fq, Fr))
        ch = OP.decision_changes(b, o)
        print("%s: single-bf16 layer vs definition: rows %.5f, columns %.5f, matches %.5f "
              "(clear: %.5f / %.5f / %.5f)" % (label, ch["row"], ch["col"], ch["matches"], ch["row_clear"],
                                               ch["col_clear"], ch["matches_clear"]))
    assert rok.mean() >= min_clear and cok.mean() >= min_clear
    np.testing.assert_array_equal(g["row_best"][rok], o["row_best"][rok])
    np.testing.assert_array_equal(g["col_best"][cok], o["col_best"][cok])
    # coarse matches: identical wherever both decisions of the pair are clear of ties
    gm = {tuple(x) for x in g["coarse"].tolist()}
    om = {tuple(x) for x in o["matches"].tolist()}
    clear = lambda ij: rok[ij[0]] and cok[ij[1]]
    assert {x for x in gm if clear(x)} == {x for x in om if clear(x)}
    assert len(om) > 0
    # probabilities of the common pairs
    gp = dict(zip(map(tuple, g["coarse"].tolist()), g["coarse_prob"]))
    for (i, j), p in zip(o["matches"].tolist(), o["prob"]):
        if (i, j) in gp:
            assert gp[(i, j)] == pytest.approx(p, rel=1e-3, abs=1e-7)
    # ascending query cells
    assert np.all(np.diff(g["coarse"][:, 0]) > 0)


def _check_fine(g, o_coarse, Fq, Fr):
    """Every coarse pair found by both sides: the window's fine matches agree on
    each query pixel whose row decision and partner-column decision are clear."""
    W = Fq.shape[2]
    Wc = W // OP.RATIO
    win = lambda pix: ((pix // W) % OP.RATIO) * OP.RATIO + (pix % W) % OP.RATIO
    gby = {}
    for (k, q, r), p in zip(g["fine"].tolist(), g["fine_prob"]):
        gby.setdefault(int(g["coarse"][k, 0]), {})[win(q)] = (win(r), float(p))
    common = {tuple(x) for x in g["coarse"].tolist()} & {tuple(x) for x in o_coarse["matches"].tolist()}
    checked = 0
    for i, j in sorted(common):
        logP, _, _ = OP.log_dual_softmax(OP._window(Fq, i, Wc, OP.RATIO) @ OP._window(Fr, j, Wc, OP.RATIO).T)
        m = OP.mnn(logP)
        opair = {int(a): int(b) for a, b in m["matches"]}
        gw = gby.get(i, {})
        for a in range(OP.RATIO * OP.RATIO):
            if m["row_flag"][a] or m["col_flag"][m["row_best"][a]]:
                continue
            if a in opair:
                assert a in gw and gw[a][0] == opair[a], (i, j, a)
                assert gw[a][1] == pytest.approx(math.exp(logP[a, opair[a]]), rel=1e-3, abs=1e-7)
            else:
                assert a not in gw, (i, j, a)
            checked += 1
    assert checked > 0


def test_pmm_small_aerial(oracle, gsr):
    Fq, Fr = _maps(oracle, 61, 240, 136, 175.0)  # 30 x 17 = 510 cells: 4 x 4 tiles, the last ragged
    o = OP.coarse_pmm(Fq, Fr)
    g = _gpu(gsr, Fq, Fr)
    _check_coarse(g, o, MIN_CLEAR_SMALL, "510 cells", Fq, Fr)
    _check_fine(g, o, Fq, Fr)


def test_pmm_multi_tile(oracle, gsr):
    Fq, Fr = _maps(oracle, 62, 512, 520, 380.0, n=40000)  # 64 x 65 = 4160 cells: 33 x 33 tiles
    o = OP.coarse_pmm(Fq, Fr)
    g = _gpu(gsr, Fq, Fr)
    _check_coarse(g, o, MIN_CLEAR_SMALL, "4160 cells", Fq, Fr)


def test_pmm_self_match_and_one_cell(oracle, gsr):
    g = np.random.default_rng(6)
    F = g.standard_normal((32, 64, 80)).astype(np.float32)  # 8 x 10 cells of distinct random vectors
    res = _gpu(gsr, F, F)
    n = 80
    np.testing.assert_array_equal(res["coarse"], np.stack([np.arange(n)] * 2, 1))
    assert len(res["fine"]) == n * 64
    np.testing.assert_array_equal(res["fine"][:, 1], res["fine"][:, 2])
    one = g.standard_normal((32, 8, 8)).astype(np.float32)
    r1 = _gpu(gsr, one, one)
    np.testing.assert_array_equal(r1["coarse"], [[0, 0]])
    # P = exp(2 M' / tau - r - c) = exp(2 (M' - M) / tau) with M (tile, tensor
    # cores) and M' (the match kernel's dot) two fp32 evaluations of the same
    # cosine, a few ulp of 1 apart: 20 x 4 x 1.2e-7 ~ 1e-5
    assert r1["coarse_prob"][0] == pytest.approx(1.0, rel=2e-5)


def test_pmm_arguments(gsr):
    with pytest.raises(gsr.GsError) as e:
        gsr.Matcher(100, 64)  # not a multiple of 8
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    m = gsr.Matcher(16, 16)
    x = torch.zeros((32, 16, 16), device="cuda")
    with pytest.raises(gsr.GsError) as e:
        m.match(x, x, tau=0.01)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    m.close()


def test_pmm_wait_that_runs_out_returns_timeout(gsr):
    """A tensor-core completion wait whose poll limit runs out makes the call
    return GS_ERR_TIMEOUT (no fault, no hang); the same matcher then matches
    normally, with results identical to a fresh matcher's."""
    g = np.random.default_rng(7)
    Fq = torch.from_numpy(g.standard_normal((32, 64, 80)).astype(np.float32)).cuda()
    Fr = torch.from_numpy(g.standard_normal((32, 64, 80)).astype(np.float32)).cuda()
    m = gsr.Matcher(64, 80)
    gsr.gs_pmm_set_wait_limit(m.handle, 0)  # every first completion wait gives up at once
    with pytest.raises(gsr.GsError) as e:
        m.match(Fq, Fr)
    assert e.value.status == gsr.GS_ERR_TIMEOUT
    gsr.gs_pmm_set_wait_limit(m.handle, gsr.GS_PMM_DEFAULT_WAIT_POLLS)
    got = m.match(Fq, Fr)
    m.close()
    ref = _gpu(gsr, Fq.cpu().numpy(), Fr.cpu().numpy())
    for k in ref:
        np.testing.assert_array_equal(got[k].cpu().numpy(), ref[k], err_msg=k)
    h = gsr.gs_pmm_create(32, 8, 8)
    with pytest.raises(gsr.GsError) as e:
        gsr.gs_pmm_set_wait_limit(h, -1)
    gsr.gs_pmm_destroy(h)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG


def test_pmm_full_size_1080p(oracle, gsr):
    """1920 x 1080 feature maps (32,400 coarse cells, a 32,400 x 32,400 similarity
    matrix) rendered by the oracle from 1,000,000 Gaussians with 32 feature
    channels, reference pose against a query 2 deg / 5 m away: every coarse code
    bit for bit, every clear decision, and the fine matches of 300 coarse pairs."""
    scene = synth.aerial_scene(2, 1_000_000, feat_dim=32)
    cam = synth.aerial_camera()
    T_ref = synth.aerial_pose()
    T_q = synth.perturb_pose(T_ref, synth.rng(100), 2.0, 5.0)
    H, W = cam["height"], cam["width"]
    maps = []
    for T in (T_q, T_ref):
        r = oracle.render(scene, cam, T, geom64=True, n_threads=16)
        maps.append(np.ascontiguousarray(r["feats"].T.reshape(32, H, W).astype(np.float32)))
    Fq, Fr = maps
    o = OP.coarse_pmm_chunked(Fq, Fr)
    g = _gpu(gsr, Fq, Fr)
    _check_coarse(g, o, MIN_CLEAR_1080P, "1080p", Fq, Fr)
    sub = o["matches"][np.sort(synth.rng(8).choice(len(o["matches"]), 300, replace=False))]
    keep = np.isin(g["coarse"][:, 0], sub[:, 0])
    gsub = {"coarse": g["coarse"], "fine": g["fine"][np.isin(g["fine"][:, 0], np.nonzero(keep)[0])],
            "fine_prob": g["fine_prob"][np.isin(g["fine"][:, 0], np.nonzero(keep)[0])]}
    _check_fine(gsub, {"matches": sub}, Fq, Fr)
