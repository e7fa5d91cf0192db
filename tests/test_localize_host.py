"""Algorithm 2's Psi and consistency rule: the library's host function against
the oracle, and the oracle's rule on hand-made pose lists; no GPU."""
import math

import numpy as np
import pytest

from oracle import localize as OL
from oracle import oracle as O
from paper_2507_15683_gb300 import synth


def _rot(axis, deg):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    th = math.radians(deg)
    T = np.eye(4)
    T[:3, :3] = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    return T


def test_pose_difference_matches_the_oracle(libgsr_path):
    from paper_2507_15683_gb300 import gsr
    g = np.random.default_rng(0)
    for _ in range(200):
        T1 = synth.perturb_pose(np.eye(4), g, 180.0, 50.0)
        T2 = synth.perturb_pose(T1, g, g.uniform(0, 60), g.uniform(0, 10))
        a, d = gsr.gs_pose_difference(T1, T2)
        oa, od = O.pose_diff(T1, T2)
        assert a == pytest.approx(oa, abs=1e-9) and d == pytest.approx(od, rel=1e-12, abs=1e-12)
    # closed forms: a rotation by theta about any axis; identical poses; a half turn
    for deg in (0.0, 1e-3, 19.999, 20.0, 20.001, 90.0, 179.0, 180.0):
        T2 = _rot(g.normal(size=3), deg)
        T2[:3, 3] = [3.0, 4.0, 0.0]
        a, d = gsr.gs_pose_difference(np.eye(4), T2)
        assert a == pytest.approx(deg, abs=1e-6) and d == pytest.approx(5.0)


def test_consistency_rule_on_hand_made_rounds():
    T = np.eye(4)
    ok, ang, _ = OL.consistency([T, _rot([0, 0, 1], 5.0), _rot([0, 0, 1], 24.0)])
    assert ok and ang == pytest.approx([5.0, 19.0])  # consecutive pairs, not the first against the rest
    ok, ang, _ = OL.consistency([T, _rot([1, 0, 0], 21.0), _rot([1, 0, 0], 21.0)])
    assert not ok and ang[1] == pytest.approx(0.0, abs=1e-6)
    ok, _, _ = OL.consistency([T, _rot([0, 1, 0], 19.9999)])  # just below the threshold: kept
    assert ok
    assert OL.consistency([T])[0]
