"""Oracle pins for the keyframe strategies (Section 4.2): KF_CONST groups, KF_DIST on
translation and rotation steps, and KF_OVRLP on a fronto-parallel plane seen from
sideways-moving frames (closed-form overlap count)."""
import math

import numpy as np
import pytest

import oracle
from oracle_helpers import identity_pose, plane_depth

INTR = (60.0, 60.0, 31.5, 23.5, 64, 48)


def _tx(t):
    T = identity_pose()
    T[0, 3] = t
    return T


def _yaw(deg):
    a = math.radians(deg)
    T = identity_pose()
    T[:, :3] = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    return T


@pytest.mark.parametrize("kappa,n", [(1, 5), (4, 10), (10, 60), (7, 20)])
def test_kf_const_groups(kappa, n):
    fk, fl, g = oracle.segment(oracle.KF_CONST, (kappa,), np.stack([identity_pose()] * n))
    assert np.array_equal(fk, np.arange(n) // kappa)
    assert g == (n + kappa - 1) // kappa and not fl.any()


def test_kf_dist_translation_and_rotation_steps():
    # 1 cm per frame, threshold 4.5 cm: frames 5 apart exceed it -> groups of 5
    poses = np.stack([_tx(0.01 * f) for f in range(23)])
    fk, fl, g = oracle.segment(oracle.KF_DIST, (0.045, 1.0), poses)
    assert np.array_equal(fk, np.arange(23) // 5) and g == 5
    # 1 degree of yaw per frame, threshold 2.5 degrees -> groups of 3
    poses = np.stack([_yaw(1.0 * f) for f in range(20)])
    fk, fl, g = oracle.segment(oracle.KF_DIST, (1.0, math.radians(2.5)), poses)
    assert np.array_equal(fk, np.arange(20) // 3)
    # either distance starts a keyframe: translation every 4th frame, rotation every 3rd
    poses = []
    for f in range(12):
        T = _yaw(1.0 * f)
        T[0, 3] = 0.012 * f
        poses.append(T)
    fk, _, _ = oracle.segment(oracle.KF_DIST, (0.04, math.radians(2.5)), np.stack(poses))
    assert np.array_equal(fk, np.arange(12) // 3)


def _inside_per_row(W, s):
    """Pixels u in [0, W) of a row whose point, shifted by s >= 0 pixels, keeps its
    nearest pixel inside the image: u + s + 1/2 < W."""
    return max(0, min(W, math.ceil(W - s - 0.5)))


def test_overlap_counts_of_a_sideways_view():
    fx, fy, cx, cy, W, H = INTR
    z0 = 2.0
    for t in (0.0, 0.031, 0.25, 1.9, 2.5):
        valid, inside, marg = oracle.overlap(plane_depth(INTR, z0), _tx(t), identity_pose(), INTR)
        s = fx * float(np.float32(t)) / z0
        assert valid == W * H
        assert inside == H * _inside_per_row(W, s)
    # a keyframe facing the other way sees nothing of the frame's points
    back = identity_pose()
    back[:, :3] = np.diag([-1.0, 1.0, -1.0])
    assert oracle.overlap(plane_depth(INTR, z0), identity_pose(), back, INTR)[1] == 0
    # invalid depth is not counted
    d = plane_depth(INTR, z0)
    d[:10] = 0.0
    assert oracle.overlap(d, identity_pose(), identity_pose(), INTR)[:2] == ((H - 10) * W, (H - 10) * W)


def test_kf_ovrlp_groups_from_the_closed_form():
    fx, fy, cx, cy, W, H = INTR
    z0, step, thr = 2.0, 0.02, 0.9
    n = 40
    poses = np.stack([_tx(step * f) for f in range(n)])
    depths = np.stack([plane_depth(INTR, z0)] * n)
    fk, fl, g = oracle.segment(oracle.KF_OVRLP, (thr,), poses, INTR, depths)
    # expected: walk the frames with the closed-form ratio
    exp, kf, grp = [0], 0, 0
    for f in range(1, n):
        s = fx * (float(np.float32(step * f)) - float(np.float32(step * kf))) / z0
        if _inside_per_row(W, s) / W < thr:
            kf, grp = f, grp + 1
        exp.append(grp)
    assert np.array_equal(fk, exp) and g == grp + 1
    assert g >= 3 and not fl.any()
    # identical views never start a keyframe
    fk, _, g = oracle.segment(oracle.KF_OVRLP, (thr,), np.stack([identity_pose()] * 8), INTR,
                              np.stack([plane_depth(INTR, z0)] * 8))
    assert g == 1 and not fk.any()
