"""The numbers the paper prints for the dense stage (tests/golden/paper_values.json,
each with its citation) against the oracle, the library's defaults and its host
functions. No GPU."""
import json
import math
import os

import numpy as np
import pytest

from oracle import localize as OL
from oracle import oracle as O
from oracle import pmm as PM

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["values"]


def _val(name):
    return GOLDEN[name]["value"]


def test_coarse_grid_gives_the_printed_search_space_reduction():
    """Sec. 3.4: H_f / H_c = 8 turns an all-pairs search over fine pixels into
    one over coarse cells 8^4 = 4096 times smaller."""
    r = _val("coarse_to_fine_ratio")
    assert PM.RATIO == r
    H, W = 64, 96
    F = np.random.default_rng(0).standard_normal((32, H, W)).astype(np.float32)
    n_cells = PM.coarse_unit_means(F).shape[0]
    assert n_cells == (H // r) * (W // r)
    assert ((H * W) ** 2) // (n_cells ** 2) == _val("search_space_reduction")
    with pytest.raises(AssertionError):
        PM.coarse_unit_means(F[:, :60])  # not a multiple of the ratio


def test_fine_windows_are_the_coarse_blocks():
    """Fine matches come from w x w windows at the coarse matches: every fine
    match of a window lies inside the 8 x 8 blocks of its coarse match."""
    w = _val("fine_window")
    H, W = 32, 48
    g = np.random.default_rng(1)
    Fq = g.standard_normal((32, H, W)).astype(np.float32)
    Fr = (Fq + 0.3 * g.standard_normal((32, H, W))).astype(np.float32)
    coarse = np.asarray(PM.coarse_pmm(Fq, Fr)["matches"])
    fine = np.asarray(PM.fine_pmm(Fq, Fr, coarse)["matches"])
    Wc = W // w
    assert len(fine) > len(coarse) > 0
    for k, q, r in fine:
        assert (q // W // w) * Wc + (q % W) // w == coarse[k][0]
        assert (r // W // w) * Wc + (r % W) // w == coarse[k][1]


def _rot_z(deg):
    t = math.radians(deg)
    T = np.eye(4)
    T[:2, :2] = [[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]]
    return T


def test_consistency_threshold_and_rounds(libgsr_path):
    from paper_2507_15683_gb300 import gsr
    tau = _val("consistency_threshold_deg")
    o = gsr.gs_localize_defaults()
    assert o.n_rounds == _val("consistency_rounds")
    assert o.max_angle_deg == tau
    # Algorithm 2 rejects an angle above tau, not one equal to it
    assert OL.consistency([np.eye(4), _rot_z(tau - 1e-6)], tau)[0]
    assert not OL.consistency([np.eye(4), _rot_z(tau + 1e-6)], tau)[0]


def test_trace_clamp_keeps_the_angle_finite(libgsr_path):
    """A relative rotation whose computed trace leaves [-1, 3] by rounding gives
    the clamp's angle (0 or 180 degrees), not NaN."""
    from paper_2507_15683_gb300 import gsr
    lo, hi = _val("trace_clamp")
    assert (lo, hi) == (-1.0, 3.0)
    up = np.eye(4)
    up[:3, :3] *= 1.0 + 2.0 ** -40  # trace(R1 R2^T) = 3 (1 + 2^-40) > 3
    down = np.eye(4)
    down[:3, :3] = np.diag([-1.0, -1.0, 1.0]) @ np.diag([1.0, 1.0, -1.0]) * (1.0 + 2.0 ** -40)  # trace -3 (1 + e)
    for T2, want in ((up, 0.0), (down, 180.0)):
        a, _ = O.pose_diff(np.eye(4), T2)
        ga, _ = gsr.gs_pose_difference(np.eye(4), T2)
        assert a == want and ga == want


def test_in_image_interval_is_half_open():
    """Algorithm 1: a projection exactly on the left or top edge is in the
    image, one exactly on the right or bottom edge is not."""
    b = _val("in_image")
    cam = {"width": 16, "height": 16, "fx": 8.0, "fy": 8.0, "cx": 8.0, "cy": 8.0}
    # u = 8 x / z + 8 with z = 1: x = -1 -> u = 0, x = 1 -> u = 16 = W (same for v)
    means = np.array([[-1.0, 0.0, 1.0], [1.0, 0.0, 1.0], [0.0, -1.0, 1.0], [0.0, 1.0, 1.0]], np.float32)
    n = len(means)
    scene = {"means": means, "scales": np.full((n, 3), 0.05, np.float32),
             "quats": np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1)),
             "opacities": np.full(n, 0.9, np.float32), "sh": np.full((n, 1, 3), 0.5, np.float32), "sh_degree": 0}
    v = O.visibility(scene, cam, np.eye(4), want_grad=False)
    np.testing.assert_array_equal(v["uv"], [[0.0, 8.0], [16.0, 8.0], [8.0, 0.0], [8.0, 16.0]])
    assert list(v["M_i"]) == [b["u_min_inclusive"], b["u_max_inclusive"], b["v_min_inclusive"],
                              b["v_max_inclusive"]]
