"""GPU dense rounds with Algorithm 2's consistency check (gs_dense_localize)
against the oracle's rounds (oracle render -> oracle PMM -> oracle PnP).

The query feature map is the oracle's render at the query pose; both sides
start from the same perturbed pose and draw the same random words. Each of
the library's rounds is checked on its own inputs: the library's render and
fine matches at the round's start pose, fed to the oracle's PnP, must give the
round's pose to 1e-3 deg and 1e-2 m. The two chains are compared only by their
outcome (both converge toward the query pose, the same reliability verdict
unless an angle lies within 1e-3 deg of the threshold): one fine match
decided within rounding of a tie reshuffles every RANSAC sample of a round.
"""
import math

import numpy as np
import pytest
import torch

from oracle import localize as OL
from oracle import pnp as OP
from paper_2507_15683_gb300 import synth

pytestmark = pytest.mark.gpu


def _rot_deg(Ra, Rb):
    M = Ra @ Rb.T
    s = 0.5 * np.linalg.norm([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]])
    return math.degrees(math.atan2(s, 0.5 * (np.trace(M) - 1.0)))


def _setup(oracle, seed, T_feat_offset=None):
    scene = synth.aerial_scene(seed, 30000, extent=(0.0, 200.0, 0.0, 200.0), n_clusters=20, feat_dim=32)
    cam = synth.camera(240, 136, 175.0)
    T_q = synth.look_pose((100.0, 40.0, 60.0), 0.0, math.radians(30.0))
    T0 = synth.perturb_pose(T_q, synth.rng(seed + 1), 2.0, 3.0)
    T_feat = T_q if T_feat_offset is None else T_feat_offset
    H, W = cam["height"], cam["width"]
    rq = oracle.render(scene, cam, T_feat, geom64=True, n_threads=16)
    Fq = np.ascontiguousarray(rq["feats"].T.reshape(32, H, W).astype(np.float32))
    words = np.random.default_rng(seed + 2).integers(0, 2 ** 32, (3, 96, 3), dtype=np.uint64).astype(np.uint32)
    return scene, cam, T_q, T0, Fq, words


def _gpu(gsr, scene, cam, T0, Fq, words):
    S = gsr.Scene(scene)
    M = gsr.Matcher(cam["height"], cam["width"])
    P = gsr.PnP(cam["height"] * cam["width"], words.shape[1])
    r = gsr.dense_localize(S, M, P, cam, T0, torch.from_numpy(Fq).cuda(),
                           torch.from_numpy(words.view(np.int32)).cuda())
    S.close()
    M.close()
    P.close()
    return r


@pytest.mark.parametrize("seed", [81, 82])
def test_dense_localize_matches_the_oracle(oracle, gsr, seed):
    """Each round against the oracle on the round's own inputs, then the chained
    rounds of both sides. The chain itself is not compared pose by pose: a
    fine match decided within rounding of a tie changes the number K of
    matches with depth, and with it every RANSAC sample (index floor(w K /
    2^32)), so the two chains may pick different, equally valid hypotheses."""
    scene, cam, T_q, T0, Fq, words = _setup(oracle, seed)
    g = _gpu(gsr, scene, cam, T0, Fq, words)
    assert g["n_rounds"] == 3
    H, W = cam["height"], cam["width"]
    S = gsr.Scene(scene)
    M = gsr.Matcher(H, W)
    fq = torch.from_numpy(Fq).cuda()
    for i in range(3):
        # the round's inputs as the library forms them: render at the round's start pose, PMM
        T_start = T0 if i == 0 else g["round_T"][i - 1]
        out = S.alloc_outputs(cam, feat_dim=32)
        S.render(cam, T_start, out)
        fine = M.match(fq, out["feats"].contiguous())["fine"].cpu().numpy()
        assert len(fine) == g["n_matches"][i]
        # the oracle's PnP on those inputs gives the round's pose
        res = OP.pnp_ransac(out["depth"].cpu().numpy(), out["alpha"].cpu().numpy(), cam, T_start, fine, words[i],
                            2.0, 5)
        dr = _rot_deg(g["round_T"][i][:3, :3], res["T"][:3, :3])
        dt = float(np.linalg.norm(g["round_T"][i][:3, 3] - res["T"][:3, 3]))
        print("round %d: %d matches, %d inliers (oracle %d); pose diff to the oracle on the same inputs %.2g deg %.2g m"
              % (i, g["n_matches"][i], g["n_inliers"][i], res["n_inliers"], dr, dt))
        assert dr < 1e-3 and dt < 1e-2
    M.close()
    S.close()
    # the oracle's own chain: renders, PMM and PnP in fp64
    o = OL.localize(scene, cam, T0, Fq, words)
    for i in range(3):
        print("chained round %d: library vs oracle %.3g deg %.3g m" % (
            i, _rot_deg(g["round_T"][i][:3, :3], o["round_T"][i][:3, :3]),
            float(np.linalg.norm(g["round_T"][i][:3, 3] - o["round_T"][i][:3, 3]))))
    if all(abs(a - 20.0) > 1e-3 for a in o["angle_deg"]) and all(abs(a - 20.0) > 1e-3 for a in g["angle_deg"]):
        assert g["reliable"] == o["reliable"]
    assert g["reliable"]
    start = _rot_deg(T0[:3, :3], T_q[:3, :3]) + np.linalg.norm(T0[:3, 3] - T_q[:3, 3])
    for T in (g["T"], o["T"]):  # both chains converge toward the query
        end = _rot_deg(T[:3, :3], T_q[:3, :3]) + np.linalg.norm(T[:3, 3] - T_q[:3, 3])
        assert end < 0.2 * start
    # Algorithm 2 on the library's rounds: its angles and distances are Psi of consecutive rounds
    for i in range(2):
        a, d = oracle.pose_diff(g["round_T"][i], g["round_T"][i + 1])
        assert g["angle_deg"][i] == pytest.approx(a, abs=1e-9) and g["trans"][i] == pytest.approx(d, abs=1e-9)
    np.testing.assert_array_equal(g["T"], g["round_T"][-1])


def test_dense_localize_flags_an_inconsistent_query(oracle, gsr):
    """Query features of a view 60 m away and turned: the rounds wander, and
    Algorithm 2 must call the result unreliable on both sides."""
    T_far = synth.look_pose((40.0, 150.0, 50.0), 2.0, math.radians(10.0))
    scene, cam, T_q, T0, Fq, words = _setup(oracle, 83, T_feat_offset=T_far)
    o = OL.localize(scene, cam, T0, Fq, words)
    g = _gpu(gsr, scene, cam, T0, Fq, words)
    print("angles gpu", g["angle_deg"], "oracle", o["angle_deg"])
    assert not o["reliable"] and not g["reliable"]


def test_dense_localize_arguments(gsr):
    cam = synth.camera(64, 48, 50.0)
    plain = synth.tiny_scene(1, n=100)
    S = gsr.Scene(plain)  # no features
    M = gsr.Matcher(48, 64)
    P = gsr.PnP(64 * 48, 8)
    Fq = torch.zeros((32, 48, 64), device="cuda")
    w = torch.zeros((3, 8, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(gsr.GsError) as e:
        gsr.dense_localize(S, M, P, cam, np.eye(4), Fq, w)
    assert e.value.status == gsr.GS_ERR_INVALID_ARG
    S.close()
    feat = synth.aerial_scene(1, 200, feat_dim=32)
    S = gsr.Scene(feat)
    with pytest.raises(gsr.GsError):  # matcher of another size
        gsr.dense_localize(S, gsr.Matcher(40, 64), P, cam, np.eye(4), Fq, w)
    with pytest.raises(gsr.GsError):  # too many rounds
        gsr.dense_localize(S, M, P, cam, np.eye(4), Fq, w, n_rounds=9)
    S.close()
    M.close()
    P.close()
