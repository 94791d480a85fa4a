"""Oracle pins for the adjoint with a given cotangent dL/dD (the vector-Jacobian product of
the keyframe integrations; an extension with no counterpart in the paper) and for the
decision-margin bookkeeping the parity tests rely on (value-changing marginal decisions
counted per voxel, Section 3 running average and Eq. 2)."""
import numpy as np

import oracle
from oracle_helpers import identity_pose, plane_depth, uniform_rgba
from paper_1709_03763_b300 import synthetic

# pixel centres placed so that no voxel of the planes below projects within 0.03 px of a
# rounding tie (u + 1/2 = 30 i / k + 15.75 has fractional parts 0.75 + j/14, 0.75 + j/6)
INTR = (30.0, 30.0, 15.25, 11.25, 32, 24)
S, MU = oracle.f32(0.02), oracle.f32(0.08)


def _cotangent(ex, seed=0):
    """A seeded cotangent on the observed voxels (input construction only)."""
    g = np.random.default_rng(seed).standard_normal(ex.W.shape)
    return ex.coords, np.where(ex.W > 0, g, 0.0)


def test_mu_is_four_voxels_and_planes_sit_on_voxel_layers():
    # the constructions below rely on exact float32 multiples of the voxel size
    assert float(np.float32(4 * S)) == MU
    assert float(np.float32(32 * S)) == 32 * S


def test_clamp_kink_is_not_counted_and_band_edge_is():
    """Fronto-parallel plane at z0 = 32 s: voxel layer 28 sits exactly on the clamp kink
    (eta = mu, where d = min(eta, mu) is continuous: not counted), layer 36 exactly on the
    band edge (eta = -mu, where the voxel is updated or not: counted once per sample)."""
    z0 = float(np.float32(32 * S))
    V = oracle.Volume(S, MU)
    V.integrate(0, plane_depth(INTR, z0), uniform_rgba(INTR, (5, 5, 5)), INTR, identity_pose())
    e = V.export()
    l = np.arange(512)
    iz = e.coords[:, 2:3].astype(np.int64) * 8 + (l // 64)[None]
    obs = e.W > 0
    assert (obs & (iz == 28)).sum() > 100 and (obs & (iz == 36)).sum() > 100
    assert np.all(e.vflag[obs & (iz == 28)] == 0)
    kf = V.kink_flags()
    assert np.all(kf[obs & (iz == 28)] == 1) and np.all(kf[obs & (iz != 28)] == 0)
    assert np.all(e.vflag[obs & (iz == 36)] == 1)
    # layers 27 and 29: 30 i / k never puts u + 1/2 within the margin of a tie
    assert np.all(e.vflag[obs & ((iz == 27) | (iz == 29))] == 0)
    # counts add up over integrations: a second keyframe with the same view doubles them
    V.integrate(1, plane_depth(INTR, z0), uniform_rgba(INTR, (5, 5, 5)), INTR, identity_pose())
    e2 = V.export()
    assert np.array_equal(e2.vflag, 2 * e.vflag)
    n_proj, n_marg = V.stats()
    assert n_marg == int(e2.vflag.sum()) and n_proj > n_marg
    # de-integration (Eq. 2) re-takes the same decisions and removes them again
    V.deintegrate(1, plane_depth(INTR, z0), uniform_rgba(INTR, (5, 5, 5)), INTR, identity_pose())
    assert np.array_equal(V.export().vflag, e.vflag)


def test_marginal_rounding_rate_matches_the_margin():
    """With fractional pixel coordinates spread uniformly, a sample is rounding-marginal
    with probability 4 tau_px (two axes, both sides of the tie); the band edge adds about
    2 tau_m per voxel spacing along the ray.  Checked on the 10-keyframe room with its
    cameras moved off the voxel lattice: there, a camera centre on a lattice plane puts
    that plane's voxels exactly on a rounding tie (u = cx), a degenerate case the parity
    tests flag but that the uniform-rate estimate does not describe."""
    w = synthetic.workload_tiny()
    V = oracle.Volume(w.voxel_size, w.trunc)
    it = w.intr.as_tuple()
    off = np.array([0.0037, 0.0051, 0.0023], np.float32)
    for k in range(10):
        T = w.kf_poses[k].copy()
        T[:, 3] += off
        V.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, T)
    n_proj, n_marg = V.stats()
    tau_px, tau_m = 5e-4, 2e-6
    expect = 4 * tau_px + 2 * tau_m / w.voxel_size
    rate = n_marg / n_proj
    assert n_proj > 500_000
    assert 0.85 * 4 * tau_px < rate < 1.15 * expect, (rate, expect)


def _plane_setup():
    z0 = 1.0047
    V = oracle.Volume(S, MU)
    d = plane_depth(INTR, z0)
    V.integrate(0, d, uniform_rgba(INTR, (1, 1, 1)), INTR, identity_pose())
    return V, d


def test_plane_adjoint_closed_forms():
    """Fronto-parallel plane at identity: d = Z(x) - z_c, so moving the camera along its
    axis by delta changes every unclamped d by +delta, as raising every depth pixel by
    delta does (grad rho_z = sum_x grad Z(x)); sideways motion and roll change no d
    (grad rho_x = grad rho_y = grad omega_z = 0)."""
    V, d = _plane_setup()
    gc, gv = _cotangent(V.export(), 3)
    gx, gd, ex, ed = V.adjoint([0], d[None], identity_pose()[None], INTR, gc, gv)
    assert abs(gx[0, 2] - gd[0].sum()) <= 1e-12 * np.abs(gd[0]).sum()
    assert gx[0, 0] == 0.0 and gx[0, 1] == 0.0 and gx[0, 5] == 0.0
    assert np.abs(gx[0, 2]) > 0 and np.abs(gx[0, 3]) > 0
    # G = 1 on every voxel: each unclamped sample adds 1 / W = 1 to its pixel
    ones = np.where(V.export().W > 0, 1.0, 0.0)
    _, g1, _, _ = V.adjoint([0], d[None], identity_pose()[None], INTR, gc, ones)
    # 8 voxel layers lie in the unclamped band [z0 - mu, z0 + mu) of each pixel ray; a
    # pixel collects every voxel of a layer whose nearest pixel it is
    assert set(np.unique(g1[0])) <= set(range(0, 40))
    assert g1[0].sum() > 0


def test_adjoint_equals_central_differences_of_its_functional():
    w = synthetic.workload_tiny()
    it = w.intr.as_tuple()
    V = oracle.Volume(w.voxel_size, w.trunc)
    for k in range(3):
        V.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    gc, gv = _cotangent(V.export(), 5)
    ids = [0, 1, 2]
    gx, gd, ex, ed = V.adjoint(ids, w.kf_depth[ids], w.kf_poses[ids], it, gc, gv)
    eps = 1e-5
    for k in ids:
        fd = np.zeros(6)
        for j in range(6):
            e = np.zeros(6)
            e[j] = eps
            fd[j] = (V.adjoint_functional(k, w.kf_depth[k], w.kf_poses[k], it, e, gc, gv)
                     - V.adjoint_functional(k, w.kf_depth[k], w.kf_poses[k], it, -e, gc, gv)) / (2 * eps)
        assert np.abs(gx[k] - fd).max() <= 1e-7 * np.abs(fd).max(), (k, gx[k], fd)
        # depth pixels: the functional is linear in one pixel's depth
        q = np.flatnonzero(np.abs(gd[k]) > 0)[:5]
        for p in q:
            f1 = V.adjoint_functional(k, w.kf_depth[k], w.kf_poses[k], it, np.zeros(6), gc, gv, pix=p, dz=1e-3)
            assert abs(f1 / 1e-3 - gd[k].flat[p]) <= 1e-9 * abs(gd[k].flat[p]) + 1e-12


def test_adjoint_agrees_with_the_loss_gradient_of_the_regulariser():
    """With no loss points, L = lambda sum W D^2 / sum W, so dL/dD = 2 lambda W D / sum W;
    the adjoint of that cotangent equals the loss gradient (two separate code paths)."""
    w = synthetic.workload_tiny()
    it = w.intr.as_tuple()
    V = oracle.Volume(w.voxel_size, w.trunc)
    for k in range(3):
        V.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    e = V.export()
    lam = 0.1
    G = 2 * lam * e.W * e.D / e.W.sum()
    ids = [0, 1, 2]
    ga, gda, _, _ = V.adjoint(ids, w.kf_depth[ids], w.kf_poses[ids], it, e.coords, G)
    gl, gdl = V.grad(ids, w.kf_depth[ids], w.kf_poses[ids], it, np.zeros((0, 3)), lam)
    assert np.abs(ga - gl).max() <= 1e-12 * np.abs(gl).max()
    assert np.abs(gda - gdl).max() <= 1e-12 * np.abs(gdl).max()


def test_adjoint_budget_vanishes_without_margins_and_covers_every_pixel_with_wide_ones():
    V, d = _plane_setup()
    gc, gv = _cotangent(V.export(), 7)
    try:
        oracle.set_margins(0.0, 0.0, 0.0)
        _, _, ex, ed = V.adjoint([0], d[None], identity_pose()[None], INTR, gc, gv)
        assert not ex.any() and not ed.any()
        # every rounding marginal: each contributing pixel carries a depth budget
        oracle.set_margins(0.5, 2e-6, 1e-6)
        _, gd, ex, ed = V.adjoint([0], d[None], identity_pose()[None], INTR, gc, gv)
        assert np.all(ed[0][gd[0] != 0] > 0)
    finally:
        oracle.set_margins()
