"""Oracle pins for the voxel-hashed TSDF: allocation, integration (running average,
Section 3 "SDF volume") and de-integration (Eq. 2, Section 4.3)."""
import numpy as np
import pytest

import oracle
from oracle_helpers import (identity_pose, plane_depth, sphere_depth, sphere_hit_z, uniform_rgba,
                            voxel_positions)

INTR = (30.0, 30.0, 15.5, 11.5, 32, 24)


def _proj(p, intr):
    fx, fy, cx, cy, W, H = intr
    return fx * p[..., 0] / p[..., 2] + cx, fy * p[..., 1] / p[..., 2] + cy


def test_plane_closed_form_truncated_distance():
    s, mu, z0 = oracle.f32(0.01), oracle.f32(0.04), 1.0047
    V = oracle.Volume(s, mu)
    V.integrate(0, plane_depth(INTR, z0), uniform_rgba(INTR, (10, 20, 30)), INTR, identity_pose())
    e = V.export()
    assert len(e.coords) > 0
    p = voxel_positions(e.coords, s)
    z = p[..., 2]
    obs = e.W > 0
    assert set(np.unique(e.W)) <= {0.0, 1.0}
    zf = float(np.float32(z0))
    expect = np.minimum(zf - z, mu)
    assert np.abs(e.D[obs] - expect[obs]).max() < 1e-12
    assert np.all(e.C[obs] == np.array([10, 20, 30.0]))
    # every unobserved voxel is behind the band, behind the camera or outside the image
    u, v = _proj(p, INTR)
    inside = (u > -0.5 + 1e-6) & (u < INTR[4] - 0.5 - 1e-6) & (v > -0.5 + 1e-6) & (v < INTR[5] - 0.5 - 1e-6)
    missing = (~obs) & (z > 0) & inside & (zf - z > -mu + 1e-9)
    assert not missing.any()
    # observed voxels are in front of / within the band
    assert np.all(zf - z[obs] >= -mu - 1e-12)


def test_sphere_closed_form_truncated_distance():
    s, mu = oracle.f32(0.01), oracle.f32(0.04)
    intr = (60.0, 60.0, 31.5, 23.5, 64, 48)
    c, r = (0.05, -0.03, 1.5), 0.4
    depth = sphere_depth(intr, c, r)
    V = oracle.Volume(s, mu)
    V.integrate(0, depth, uniform_rgba(intr, (1, 2, 3)), intr, identity_pose())
    e = V.export()
    p = voxel_positions(e.coords, s)
    obs = (e.W > 0) & (e.vflag == 0)
    u, v = _proj(p, intr)
    pu, pv = np.floor(u + 0.5), np.floor(v + 0.5)
    # the ray through that pixel's centre, intersected with the sphere in closed form
    d = np.stack([(pu - intr[2]) / intr[0], (pv - intr[3]) / intr[1], np.ones_like(pu)], -1)
    zhit = sphere_hit_z(d, c, r)
    expect = np.minimum(zhit - p[..., 2], mu)
    err = np.abs(e.D[obs] - expect[obs])
    # depth image is stored as float32: 1e-7 relative at 1.1-1.9 m
    assert err.max() < 5e-7, err.max()
    assert obs.sum() > 1000


def _run(kf_list, tiny, rgba8=False):
    V = oracle.Volume(tiny.voxel_size, tiny.trunc, rgba8=rgba8)
    for k in kf_list:
        V.integrate(int(k), tiny.kf_depth[k], tiny.kf_rgba[k], tiny.intr.as_tuple(), tiny.kf_poses[k])
    return V


def _as_dict(e):
    return {tuple(c): i for i, c in enumerate(e.coords)}


def test_integrate_then_deintegrate_restores(tiny):
    it = tiny.intr.as_tuple()
    V = _run(range(10), tiny)
    V.deintegrate(4, tiny.kf_depth[4], tiny.kf_rgba[4], it, tiny.kf_poses[4])
    ref = _run([k for k in range(10) if k != 4], tiny)
    a, b = V.export(), ref.export()
    ia, ib = _as_dict(a), _as_dict(b)
    assert set(ib) <= set(ia)
    common = [(ia[k], ib[k]) for k in ib]
    A = np.array([x for x, _ in common])
    B = np.array([y for _, y in common])
    assert np.array_equal(a.W[A], b.W[B])
    assert np.abs(a.D[A] - b.D[B]).max() < 1e-12
    assert np.abs(a.C[A] - b.C[B]).max() < 1e-9
    extra = np.array([ia[k] for k in ia if k not in ib])
    assert len(extra) > 0
    assert np.all(a.W[extra] == 0) and np.all(a.D[extra] == 0) and np.all(a.C[extra] == 0)


def test_single_integrate_deintegrate_empties_volume(tiny):
    it = tiny.intr.as_tuple()
    V = _run([3], tiny)
    assert (V.export().W > 0).sum() > 10000
    V.deintegrate(3, tiny.kf_depth[3], tiny.kf_rgba[3], it, tiny.kf_poses[3])
    e = V.export()
    assert np.all(e.W == 0) and np.all(e.D == 0) and np.all(e.C == 0)


def test_weights_count_identical_observations(tiny):
    it = tiny.intr.as_tuple()
    one = _run([2], tiny).export()
    V = oracle.Volume(tiny.voxel_size, tiny.trunc)
    for kid in range(3):
        V.integrate(kid, tiny.kf_depth[2], tiny.kf_rgba[2], it, tiny.kf_poses[2])
    three = V.export()
    assert np.array_equal(one.coords, three.coords)
    assert np.array_equal(three.W, 3 * one.W)
    obs = one.W > 0
    assert np.abs(three.D[obs] - one.D[obs]).max() < 1e-12


def test_integration_order_invariance(tiny):
    a = _run([1, 5, 8], tiny).export()
    b = _run([8, 1, 5], tiny).export()
    assert np.array_equal(a.coords, b.coords)
    assert np.array_equal(a.W, b.W)
    assert np.abs(a.D - b.D).max() < 1e-12
    assert np.abs(a.C - b.C).max() < 1e-9


def test_rgba8_rounds_half_to_even():
    s, mu, z0 = 0.01, 0.04, 1.0047
    for c1, c2, expect in [(10, 13, 12), (10, 11, 10), (11, 12, 12), (200, 201, 200)]:
        V = oracle.Volume(s, mu, rgba8=True)
        V.integrate(0, plane_depth(INTR, z0), uniform_rgba(INTR, (c1, c1, c1)), INTR, identity_pose())
        V.integrate(1, plane_depth(INTR, z0), uniform_rgba(INTR, (c2, c2, c2)), INTR, identity_pose())
        e = V.export()
        obs = e.W == 2
        assert obs.sum() > 0
        assert np.all(e.C[obs] == expect), (c1, c2)


def test_weight_reaching_zero_resets_voxel():
    s, mu, z0 = 0.01, 0.04, 1.0047
    d = plane_depth(INTR, z0)
    V = oracle.Volume(s, mu)
    V.integrate(0, d, uniform_rgba(INTR, (9, 9, 9)), INTR, identity_pose())
    V.integrate(1, d, uniform_rgba(INTR, (3, 3, 3)), INTR, identity_pose())
    V.deintegrate(0, d, uniform_rgba(INTR, (9, 9, 9)), INTR, identity_pose())
    e = V.export()
    obs = e.W == 1
    assert np.all(e.C[obs] == 3.0)
    V.deintegrate(1, d, uniform_rgba(INTR, (3, 3, 3)), INTR, identity_pose())
    e = V.export()
    assert np.all(e.W == 0) and np.all(e.D == 0) and np.all(e.C == 0)


def _segment_blocks(depth, pose, intr, s, mu, n_samples=2001, delta=0.0):
    fx, fy, cx, cy, W, H = intr
    B = 8 * s
    R = pose[:, :3].astype(np.float64)
    t = pose[:, 3].astype(np.float64)
    out = set()
    ts = np.linspace(0.0, 1.0, n_samples)
    offs = [np.zeros(3)] if delta == 0 else [np.array([a, b, c]) for a in (-delta, delta)
                                              for b in (-delta, delta) for c in (-delta, delta)]
    for v in range(H):
        for u in range(W):
            z = float(depth[v, u])
            if z <= 0:
                continue
            ray = np.array([(u - cx) / fx, (v - cy) / fy, 1.0])
            q0 = R @ (ray * (z - mu)) + t
            q1 = R @ (ray * (z + mu)) + t
            pts = q0[None] + ts[:, None] * (q1 - q0)[None]
            for o in offs:
                out |= set(map(tuple, np.floor((pts + o) / B).astype(np.int64)))
    return out


def test_allocation_matches_dense_segment_sampling(tiny):
    # 16x12 keyframe: subsample the tiny workload's first keyframe by 20
    d = tiny.kf_depth[0].numpy()[::20, ::20].copy()
    fx = tiny.intr.fx / 20
    intr = (fx, fx, (16 - 1) / 2, (12 - 1) / 2, 16, 12)
    pose = tiny.kf_poses[0]
    s, mu = oracle.f32(tiny.voxel_size), oracle.f32(tiny.trunc)
    coords, marg = oracle.allocation_set(d, pose, intr, s, mu)
    A_all = set(map(tuple, coords))
    A_robust = set(map(tuple, coords[marg == 0]))
    step = 2 * mu / 2000
    inner = _segment_blocks(d, pose, intr, s, mu)
    outer = _segment_blocks(d, pose, intr, s, mu, delta=2 * step)
    assert inner <= A_all
    assert A_robust <= outer
    assert len(A_robust) >= 0.95 * len(inner)


def test_reintegration_batch_equals_integrating_at_updated_poses(tiny):
    """Section 4.3: de-integrating at the former pose and re-integrating at the updated
    pose leaves the volume as if the keyframes had been integrated at the updated pose."""
    it = tiny.intr.as_tuple()
    ids = [int(i) for i in tiny.update_ids]
    V = _run(range(10), tiny)
    V.reintegrate_batch(ids, tiny.kf_depth[ids], tiny.kf_rgba[ids], tiny.kf_poses[ids], tiny.new_poses[ids], it)
    ref = oracle.Volume(tiny.voxel_size, tiny.trunc)
    for k in range(10):
        pose = tiny.new_poses[k] if k in ids else tiny.kf_poses[k]
        ref.integrate(k, tiny.kf_depth[k], tiny.kf_rgba[k], it, pose)
    a, b = V.export(), ref.export()
    ia, ib = _as_dict(a), _as_dict(b)
    assert set(ib) <= set(ia)
    A = np.array([ia[k] for k in ib])
    B = np.array([ib[k] for k in ib])
    assert np.array_equal(a.W[A], b.W[B])
    assert np.abs(a.D[A] - b.D[B]).max() < 1e-12
    assert np.abs(a.C[A] - b.C[B]).max() < 1e-9
    extra = np.array([ia[k] for k in ia if k not in ib])
    assert np.all(a.W[extra] == 0) and np.all(a.D[extra] == 0)
    # the touched lists now hold the updated poses' allocation sets
    for k in ids:
        c1, _ = V.touched(k)
        c2, _ = ref.touched(k)
        assert np.array_equal(c1, c2)
