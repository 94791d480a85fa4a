"""Oracle pins for keyframe selection (Section 4.3, Eq. 3; worked example of Fig. 4)."""
import json
import math
import os

import numpy as np

import oracle
from paper_1709_03763_b300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig4_selection.json")


def test_fig4_consecutive_selection():
    g = json.load(open(GOLDEN))
    j, sums = oracle.select_consecutive(np.array(g["distances"], float), g["m"])
    assert j + 1 == g["j_star_1based"]
    assert list(sums) == g["window_sums"]
    assert [j + 1 + i for i in range(g["m"])] == g["consecutive_frames_1based"]


def test_fig4_bundlefusion_topm_ties_to_lower_index():
    g = json.load(open(GOLDEN))
    top = oracle.select_topm(np.array(g["distances"], float), g["m"])
    # frames 3 and 6 both have distance 4; the figure picks 3
    assert list(top + 1) == g["bundlefusion_top_m_1based"]


def test_consecutive_ties_pick_first_window():
    j, sums = oracle.select_consecutive(np.array([1.0, 1, 1, 1, 1, 1]), 3)
    assert j == 0 and list(sums) == [3, 3, 3, 3]


def _pose(R, t):
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T


def test_pose_distance_closed_forms():
    I = np.eye(3)
    # pure translation: scale 1 on translation
    assert math.isclose(oracle.pose_distance(_pose(I, [0, 0, 0]), _pose(I, [0.3, -0.4, 0])), 0.5, rel_tol=1e-6)
    # rotation about a single axis by a: one Euler angle changes by a, scaled by 2
    for axis in ([0, 0, 1], [0, 1, 0], [1, 0, 0]):
        a = 0.3
        R = synthetic.axis_angle(np.array(axis, float), a)
        d = oracle.pose_distance(_pose(I, [0, 0, 0]), _pose(R, [0, 0, 0]))
        assert math.isclose(d, 2 * a, rel_tol=1e-5), (axis, d)
    # yaw wrap-around: 179 deg vs -179 deg is 2 deg apart
    Ra = synthetic.axis_angle(np.array([0, 0, 1.0]), math.radians(179))
    Rb = synthetic.axis_angle(np.array([0, 0, 1.0]), math.radians(-179))
    d = oracle.pose_distance(_pose(Ra, [0, 0, 0]), _pose(Rb, [0, 0, 0]))
    assert math.isclose(d, 2 * math.radians(2), rel_tol=1e-4)
    # combined: rotation and translation add in quadrature
    R = synthetic.axis_angle(np.array([0, 0, 1.0]), 0.1)
    d = oracle.pose_distance(_pose(I, [0, 0, 0]), _pose(R, [0, 0, 0.2]))
    assert math.isclose(d, math.hypot(0.2, 0.2), rel_tol=1e-5)
