"""Oracle pins for the loss on the fused SDF and its gradient with respect to keyframe
se(3) poses and depth pixels (an extension with no counterpart in the paper)."""
import numpy as np

import oracle
from oracle_helpers import identity_pose, plane_depth, uniform_rgba
from paper_1709_03763_b300 import synthetic

INTR = (30.0, 30.0, 15.5, 11.5, 32, 24)
S, MU = oracle.f32(0.01), oracle.f32(0.04)


def _plane_points(z, n=3000, seed=0):
    g = np.random.default_rng(seed)
    x = g.uniform(-0.45, 0.45, n) * z
    y = g.uniform(-0.33, 0.33, n) * z
    return np.stack([x, y, np.full(n, z)], 1)


def _plane_volume(zdepth):
    V = oracle.Volume(S, MU)
    V.integrate(0, plane_depth(INTR, zdepth), uniform_rgba(INTR, (1, 1, 1)), INTR, identity_pose())
    return V


def test_plane_moved_along_optical_axis_closed_form():
    # z0 and z0 +- eps are exact float32 values, so the central difference is centred
    # exactly on the analytic evaluation point
    z0, eps = float(np.float32(1.0047)), 2.0 ** -13
    pts = _plane_points(1.02)
    V = _plane_volume(z0)
    gx, gd = V.grad([0], plane_depth(INTR, z0)[None], identity_pose()[None], INTR, pts)
    zp, zm = np.float32(z0 + eps), np.float32(z0 - eps)
    assert float(zp) - z0 == eps and z0 - float(zm) == eps
    Vp, Vm = _plane_volume(zp), _plane_volume(zm)
    ep, em = Vp.export(), Vm.export()
    # no discrete decision changes between the two shifted planes
    assert np.array_equal(ep.coords, em.coords) and np.array_equal(ep.W, em.W)
    Lp, np_, _ = Vp.loss(pts)
    Lm, nm, _ = Vm.loss(pts)
    assert np_ == nm > 0
    fd = (Lp - Lm) / (float(zp) - float(zm))
    # moving the camera forward by rho_z == moving the plane back by the same amount
    assert abs(gx[0, 2] - fd) < 1e-6 * abs(fd), (gx[0, 2], fd)
    # shifting every depth pixel by the same amount is the same motion
    assert abs(gd.sum() - fd) < 1e-6 * abs(fd)
    # a fronto-parallel plane at identity: roll about the optical axis and sideways
    # motion do not change any z-distance
    assert gx[0, 5] == 0.0 and gx[0, 0] == 0.0 and gx[0, 1] == 0.0


def test_analytic_gradient_matches_frozen_central_differences(tiny):
    it = tiny.intr.as_tuple()
    V = oracle.Volume(tiny.voxel_size, tiny.trunc)
    for k in range(10):
        V.integrate(k, tiny.kf_depth[k], tiny.kf_rgba[k], it, tiny.kf_poses[k])
    pts = synthetic.surface_points(tiny.scene, 20000, 1)
    L, nv, _ = V.loss(pts)
    assert nv > 2000
    kfs = [0, 4, 7]
    gx, gd = V.grad(kfs, tiny.kf_depth[kfs], tiny.kf_poses[kfs], it, pts)
    eps = 1e-4

    def central(f):
        # fourth-order central difference: truncation error O(eps^4)
        return (8 * (f(eps) - f(-eps)) - (f(2 * eps) - f(-2 * eps))) / (12 * eps)

    for row, k in enumerate(kfs):
        fd = np.zeros(6)
        for j in range(6):
            e = np.eye(6)[j]
            fd[j] = central(lambda h: V.loss_perturbed(k, tiny.kf_depth[k], tiny.kf_poses[k], it, h * e, pts))
        scale = np.abs(fd).max()
        assert scale > 0
        assert np.abs(gx[row] - fd).max() < 1e-8 * scale, (k, gx[row], fd)
        # depth pixels: the few with the largest gradient (the loss is exactly quadratic in them)
        flat = np.argsort(-np.abs(gd[row]).ravel())[:4]
        for pix in flat:
            f = central(lambda h: V.loss_perturbed(k, tiny.kf_depth[k], tiny.kf_poses[k], it, np.zeros(6), pts,
                                                   pix=int(pix), dz=h))
            assert abs(gd[row].ravel()[pix] - f) < 1e-8 * abs(f) + 1e-15, (k, pix)


def test_zero_perturbation_reproduces_loss(tiny):
    it = tiny.intr.as_tuple()
    V = oracle.Volume(tiny.voxel_size, tiny.trunc)
    for k in range(3):
        V.integrate(k, tiny.kf_depth[k], tiny.kf_rgba[k], it, tiny.kf_poses[k])
    pts = synthetic.surface_points(tiny.scene, 5000, 1)
    L, _, _ = V.loss(pts)
    L0 = V.loss_perturbed(1, tiny.kf_depth[1], tiny.kf_poses[1], it, np.zeros(6), pts)
    assert abs(L - L0) < 1e-14 * max(1.0, abs(L))


def test_loss_of_exact_plane_volume():
    # points on the plane sit where the (linear, unclamped) distance field is zero
    z0 = 1.0047
    V = _plane_volume(z0)
    pts = _plane_points(float(np.float32(z0)), 500)
    L, nv, _ = V.loss(pts, lam=0.0)
    assert nv == 500
    assert L < 1e-24
