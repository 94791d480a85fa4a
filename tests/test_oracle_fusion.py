"""Oracle pins for keyframe depth fusion, Eq. 1 (Section 3 "Keyframe Fusion")."""
import math

import numpy as np

import oracle
from oracle_helpers import identity_pose, plane_depth

INTR = (30.0, 30.0, 15.5, 11.5, 32, 24)


def _interior(shape):
    m = np.zeros(shape, bool)
    m[1:-1, 1:-1] = True
    return m


def test_identical_frames_fuse_to_same_depth_and_summed_weight():
    z0 = 1.37
    kappa = 4
    d = np.stack([plane_depth(INTR, z0)] * kappa)
    poses = np.stack([identity_pose()] * kappa)
    Z, W, fl = oracle.fuse(d, poses, identity_pose(), INTR)
    m = _interior(Z.shape)
    zf = float(np.float32(z0))
    assert np.abs(Z[m] - zf).max() < 1e-12
    # fronto-parallel plane: cos(theta) = 1, w_z = Z^-2 per frame
    assert np.abs(W[m] - kappa / zf ** 2).max() < 1e-9
    assert np.all(W[~m] == 0)


def test_tilted_plane_weight_is_cos_theta_over_z_squared():
    fx, fy, cx, cy, Wd, H = INTR
    tilt = math.radians(35.0)
    n = np.array([0.0, math.sin(tilt), -math.cos(tilt)])   # plane n . p = -d0
    d0 = 1.2
    v, u = np.mgrid[0:H, 0:Wd].astype(np.float64)
    ray = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1)
    z = (-d0 / (ray @ n))
    depth = z.astype(np.float32)
    Z, W, fl = oracle.fuse(depth[None], identity_pose()[None], identity_pose(), INTR)
    m = _interior(Z.shape)
    zf = depth.astype(np.float64)
    # depth is float32: the estimated normal matches the plane's to ~1e-6
    assert np.abs(W[m] - math.cos(tilt) / zf[m] ** 2).max() < 1e-4 * W[m].max()
    assert np.abs(Z[m] - zf[m]).max() < 1e-12


def test_translated_views_of_plane_fuse_to_plane_depth():
    z0 = 2.1
    poses = []
    for k in range(5):
        T = identity_pose()
        T[0, 3] = 0.013 * k
        poses.append(T)
    d = np.stack([plane_depth(INTR, z0)] * 5)
    Z, W, fl = oracle.fuse(d, np.stack(poses), identity_pose(), INTR)
    cov = W > 0
    assert cov.sum() > 0.8 * Z.size
    assert np.abs(Z[cov] - float(np.float32(z0))).max() < 1e-6


def test_eq1_order_invariance(tiny):
    frames = tiny.kf_depth[[0, 1, 9]].numpy()
    poses = tiny.kf_poses[[0, 1, 9]]
    it = tiny.intr.as_tuple()
    Za, Wa, _ = oracle.fuse(frames, poses, poses[0], it)
    Zb, Wb, _ = oracle.fuse(frames[::-1].copy(), poses[::-1].copy(), poses[0], it)
    assert np.abs(Wa - Wb).max() < 1e-9 * Wa.max()
    m = Wa > 0
    assert np.abs(Za[m] - Zb[m]).max() < 1e-12
    assert m.sum() > 0.5 * m.size


def test_keyframe_frame_alone_is_reproduced(tiny):
    d = tiny.kf_depth[3].numpy()
    it = tiny.intr.as_tuple()
    Z, W, fl = oracle.fuse(d[None], tiny.kf_poses[3][None], tiny.kf_poses[3], it)
    m = (W > 0) & (fl == 0)
    assert m.sum() > 0.8 * (d > 0).sum()
    assert np.abs(Z[m] - d[m]).max() < 1e-6


def test_depth_discontinuity_pixels_are_dropped():
    fx, fy, cx, cy, Wd, H = INTR
    d = plane_depth(INTR, 1.0)
    d[:, 16:] = 1.5           # step edge between columns 15 and 16
    d[5, 5] = 0.0             # an invalid pixel: its 4 neighbours are dropped
    Z, W, fl = oracle.fuse(d[None], identity_pose()[None], identity_pose(), INTR, disc_rel=0.1)
    assert np.all(W[1:-1, 15] == 0) and np.all(W[1:-1, 16] == 0)
    assert np.all(W[1:-1, 14] > 0) and np.all(W[1:-1, 17] > 0)
    assert W[5, 5] == 0 and W[4, 5] == 0 and W[6, 5] == 0 and W[5, 4] == 0 and W[5, 6] == 0
    # a small relative step below the threshold is kept
    d2 = plane_depth(INTR, 1.0)
    d2[:, 16:] = 1.05
    Z2, W2, _ = oracle.fuse(d2[None], identity_pose()[None], identity_pose(), INTR, disc_rel=0.1)
    assert np.all(W2[1:-1, 15] > 0)
