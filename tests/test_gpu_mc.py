"""GPU Marching Cubes (Section 3 "SDF volume") and block import against the oracle on
identical block arrays: an analytic sphere, an oracle-integrated Kinect-style volume,
missing neighbours and unobserved voxels, empty volumes and a short output buffer."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_03763_b300 import SurfcorrError, Volume, synthetic

pytestmark = pytest.mark.gpu

POS_TOL = 2e-6  # metres: float32 vertex arithmetic on coordinates of a few metres


def _sphere_blocks(s, c, r, lo, hi):
    coords = np.array([[x, y, z] for z in range(lo[2], hi[2]) for y in range(lo[1], hi[1])
                       for x in range(lo[0], hi[0])], np.int32)
    v = np.array([[i % 8, (i // 8) % 8, i // 64] for i in range(512)])
    P = (coords[:, None, :] * 8 + v[None]) * s
    D = (np.linalg.norm(P - c, axis=-1) - r).astype(np.float32)
    W = np.ones_like(D)
    return coords, D, W


def _gpu_mesh(s, coords, D, W, colour="rgba8", C=None):
    V = Volume(s, 4 * s, 1 << 12, max_blocks=max(len(coords), 1) + 64, colour=colour, max_keyframes=4)
    if len(coords):
        V.import_blocks(torch.from_numpy(coords).cuda(), torch.from_numpy(D).cuda(), torch.from_numpy(W).cuda(),
                        None if C is None else torch.from_numpy(C).cuda())
    tri, cube = V.marching_cubes(cubes=True)
    torch.cuda.synchronize()
    out = tri.cpu().numpy().astype(np.float64), cube.cpu().numpy()
    V.close()
    return out


def _match(tri_g, cube_g, tri_o, cube_o):
    """Same triangles: identical cube ids (x, y, z, k) and vertex positions within POS_TOL."""
    assert len(tri_g) == len(tri_o)
    kg = np.lexsort(cube_g.T[::-1])
    ko = np.lexsort(cube_o.T[::-1])
    assert np.array_equal(cube_g[kg], cube_o[ko])
    err = np.abs(tri_g[kg] - tri_o[ko])
    scale = np.maximum(1.0, np.abs(tri_o[ko]))
    assert (err / scale).max() <= POS_TOL, float(err.max())


def test_sphere_matches_oracle():
    s = float(np.float32(0.01))
    c = np.array([0.1601, 0.1593, 0.1612])
    coords, D, W = _sphere_blocks(s, c, 0.107, (0, 0, 0), (4, 4, 4))
    tri_g, cube_g = _gpu_mesh(s, coords, D, W)
    tri_o, cube_o = oracle.marching_cubes(coords, D, W, s)
    assert len(tri_o) > 1000
    _match(tri_g, cube_g, tri_o, cube_o)


def test_oracle_volume_matches_oracle_mc():
    # a Kinect-style volume made by the oracle (three keyframes of the tiny room),
    # rounded to float32 and loaded into the GPU volume
    w = synthetic.workload_tiny()
    O = oracle.Volume(w.voxel_size, w.trunc)
    for k in range(3):
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], w.intr.as_tuple(), w.kf_poses[k])
    ex = O.export()
    coords = ex.coords.astype(np.int32)
    D = ex.D.astype(np.float32)
    W = ex.W.astype(np.float32)
    C = np.ascontiguousarray(np.transpose(ex.C, (0, 2, 1)).astype(np.float32))  # [n,3,512]
    tri_g, cube_g = _gpu_mesh(oracle.f32(w.voxel_size), coords, D, W, colour="f32", C=C)
    tri_o, cube_o = oracle.marching_cubes(coords, D, W, w.voxel_size)
    assert len(tri_o) > 10000
    _match(tri_g, cube_g, tri_o, cube_o)


def test_missing_neighbours_and_unobserved_voxels():
    s = float(np.float32(0.02))
    c = np.array([0.08, 0.08, 0.08])
    coords, D, W = _sphere_blocks(s, c, 0.1, (-1, -1, -1), (2, 2, 2))
    keep = np.ones(len(coords), bool)
    keep[[3, 11, 20]] = False            # holes in the block grid
    W[5, :200] = 0.0                     # unobserved voxels
    W[7, ::3] = 0.0
    coords, D, W = coords[keep], D[keep], W[keep]
    tri_g, cube_g = _gpu_mesh(s, coords, D, W)
    tri_o, cube_o = oracle.marching_cubes(coords, D, W, s)
    assert len(tri_o) > 0
    _match(tri_g, cube_g, tri_o, cube_o)


def test_empty_volume_and_short_buffer():
    s = float(np.float32(0.01))
    tri, cube = _gpu_mesh(s, np.zeros((0, 3), np.int32), None, None)
    assert len(tri) == 0
    c = np.array([0.1601, 0.1593, 0.1612])
    coords, D, W = _sphere_blocks(s, c, 0.107, (0, 0, 0), (4, 4, 4))
    V = Volume(s, 4 * s, 1 << 12, max_blocks=256, max_keyframes=4)
    V.import_blocks(torch.from_numpy(coords).cuda(), torch.from_numpy(D).cuda(), torch.from_numpy(W).cuda())
    full = V.marching_cubes()
    with pytest.raises(SurfcorrError):
        V.marching_cubes(capacity=len(full) // 2)
    # importing the same blocks again overwrites them: same mesh
    V.import_blocks(torch.from_numpy(coords).cuda(), torch.from_numpy(D).cuda(), torch.from_numpy(W).cuda())
    again = V.marching_cubes()
    assert len(again) == len(full) and V.info()["allocated_blocks"] == len(coords)
    V.close()


def test_mesh_of_a_gpu_integrated_volume():
    # the full GPU path: integrate keyframes, then mesh; every vertex lies in its cube and
    # each cube's corners are observed voxels of the extracted volume
    w = synthetic.workload_tiny()
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, max_blocks=1 << 16, max_keyframes=8)
    for k in range(3):
        V.integrate(k, w.kf_depth[k].cuda(), w.kf_rgba[k].cuda(), w.intr, w.kf_poses[k])
    tri, cube = V.marching_cubes(cubes=True)
    tri, cube = tri.cpu().numpy().astype(np.float64), cube.cpu().numpy()
    s = oracle.f32(w.voxel_size)
    assert len(tri) > 10000
    lo = cube[:, None, :3] * s
    assert np.all(tri >= lo - 1e-5) and np.all(tri <= lo + s + 1e-5)
    ex = V.extract()
    key = {tuple(c): i for i, c in enumerate(ex["coords"].cpu().numpy())}
    Wv = ex["W"].cpu().numpy()
    for x, y, z, _ in cube[:: max(1, len(cube) // 500)]:
        for i in range(8):
            vx, vy, vz = x + (i & 1), y + ((i >> 1) & 1), z + ((i >> 2) & 1)
            b = key[(vx // 8, vy // 8, vz // 8)]
            assert Wv[b, (vx % 8) + 8 * (vy % 8) + 64 * (vz % 8)] > 0
    V.close()
