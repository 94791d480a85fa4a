"""Oracle pins for Marching Cubes iso-surface extraction (Section 3 "SDF volume"):
closed-form cases of the triangulation rule, a plane (exact vertices, area,
orientation, skipped boundary cubes) and a sphere (vertex distance bound, closed
orientable genus-0 mesh, enclosed volume)."""
import math

import numpy as np
import pytest

import oracle

CORNER = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)])


def _edge_corners(e):
    """Corners (lo, hi) of cube edge e, found geometrically: the edge along axis e // 4
    whose other two coordinates are the bits of e % 4 (lower axis first)."""
    a = e // 4
    others = [d for d in range(3) if d != a]
    lo = np.zeros(3, int)
    lo[others[0]] = (e % 4) & 1
    lo[others[1]] = ((e % 4) >> 1) & 1
    hi = lo.copy()
    hi[a] = 1
    idx = lambda p: int(p[0] + 2 * p[1] + 4 * p[2])
    return idx(lo), idx(hi)


def _midpoint(e):
    lo, hi = _edge_corners(e)
    return (CORNER[lo] + CORNER[hi]) / 2.0


def _normal(tri):
    p = [_midpoint(e) for e in tri]
    return np.cross(p[1] - p[0], p[2] - p[0])


# ------------------------------------------------------------------ the rule, per cube

@pytest.mark.parametrize("corner", range(8))
def test_single_corner_is_cut_off_facing_out(corner):
    t = oracle.mc_case(1 << corner)
    assert len(t) == 1
    # the triangle's three edges are the three edges at that corner
    assert sorted(set(c for e in t[0] for c in _edge_corners(e)) - {corner}) == \
        sorted(corner ^ (1 << a) for a in range(3))
    for e in t[0]:
        assert corner in _edge_corners(e)
    # its normal points away from the inside corner
    centre = np.mean([_midpoint(e) for e in t[0]], 0)
    assert np.dot(_normal(t[0]), centre - CORNER[corner]) > 0
    # the complement (one corner outside) gives the same triangle facing the corner
    t2 = oracle.mc_case(255 ^ (1 << corner))
    assert len(t2) == 1 and sorted(t2[0]) == sorted(t[0])
    assert np.dot(_normal(t2[0]), centre - CORNER[corner]) < 0


@pytest.mark.parametrize("mask", [0x69, 0x96])
def test_checkerboard_cuts_every_inside_corner_separately(mask):
    t = oracle.mc_case(mask)
    assert len(t) == 4
    inside = [i for i in range(8) if (mask >> i) & 1]
    cut = []
    for tri in t:
        common = set(_edge_corners(tri[0])) & set(_edge_corners(tri[1])) & set(_edge_corners(tri[2]))
        assert len(common) == 1
        c = common.pop()
        cut.append(c)
        centre = np.mean([_midpoint(e) for e in tri], 0)
        assert np.dot(_normal(tri), centre - CORNER[c]) > 0
    assert sorted(cut) == inside


def test_half_cube_is_a_square_facing_out():
    # corners with z = 0 inside (mask 0x0f): the surface is the square z = 1/2, normal +z
    t = oracle.mc_case(0x0F)
    assert len(t) == 2
    edges = sorted(set(e for tri in t for e in tri))
    assert edges == [8, 9, 10, 11]  # the four z edges
    for tri in t:
        n = _normal(tri)
        assert n[2] > 0 and abs(n[0]) < 1e-12 and abs(n[1]) < 1e-12


def test_every_case_uses_exactly_the_crossed_edges():
    # every edge whose corners differ carries a vertex of the case, and no other edge
    for m in range(256):
        t = oracle.mc_case(m)
        crossed = {e for e in range(12) if ((m >> _edge_corners(e)[0]) & 1) != ((m >> _edge_corners(e)[1]) & 1)}
        used = {e for tri in t for e in tri}
        assert used == crossed, m
        assert len(t) <= 5


# ------------------------------------------------------------------ plane and sphere

def _blocks_for(fn, lo, hi, s):
    """Blocks lo..hi-1 (inclusive ranges per axis) with D = fn(p) and W = 1."""
    coords = np.array([[x, y, z] for z in range(lo[2], hi[2]) for y in range(lo[1], hi[1])
                       for x in range(lo[0], hi[0])], np.int32)
    v = np.array([[i % 8, (i // 8) % 8, i // 64] for i in range(512)])
    P = (coords[:, None, :] * 8 + v[None]) * s
    D = fn(P).astype(np.float32)
    W = np.ones_like(D)
    return coords, D, W


def test_plane_vertices_area_orientation_and_skipped_boundary():
    s = float(np.float32(0.01))
    z0 = 0.0437   # between voxel layers 4 and 5 of block z = 0
    nb = 2
    coords, D, W = _blocks_for(lambda P: z0 - P[..., 2], (0, 0, 0), (nb, nb, 1), s)
    tri, cube = oracle.marching_cubes(coords, D, W, s)
    # every vertex lies on the plane (D is linear in z): up to float32 D
    zD = np.abs(tri[..., 2] - z0)
    assert zD.max() < 1e-8
    # cubes need all 8 corners: the last voxel column / row of the 2 x 2 block slab has
    # no neighbour, so (8 nb - 1)^2 cubes are crossed, two triangles each
    n_cubes = (8 * nb - 1) ** 2
    assert len(tri) == 2 * n_cubes
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=-1)
    assert abs(area.sum() - n_cubes * s * s) < 1e-9
    # normals point to D > 0, i.e. towards -z
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    assert np.all(n[:, 2] < 0)
    # unobserved corners also skip cubes
    W2 = W.copy()
    W2[0, :] = 0.0
    tri2, _ = oracle.marching_cubes(coords, D, W2, s)
    assert len(tri2) < len(tri)


def _mesh_topology(tri):
    key = lambda p: tuple(np.round(p, 12))
    vid = {}
    F = []
    for t in tri:
        F.append([vid.setdefault(key(p), len(vid)) for p in t])
    edges = {}
    for f in F:
        for i in range(3):
            a, b = f[i], f[(i + 1) % 3]
            edges.setdefault((min(a, b), max(a, b)), []).append((a, b))
    return len(vid), edges, len(F)


def test_sphere_is_closed_orientable_genus0_with_bounded_error():
    s = float(np.float32(0.01))
    r = 0.107
    c = np.array([0.1601, 0.1593, 0.1612])
    coords, D, W = _blocks_for(lambda P: np.linalg.norm(P - c, axis=-1) - r, (0, 0, 0), (4, 4, 4), s)
    tri, cube = oracle.marching_cubes(coords, D, W, s)
    assert len(tri) > 1000
    # vertex distance to the sphere: linear interpolation of a function with second
    # derivative <= 1 / (r - 2 s) along an edge of length s errs by <= s^2 / (8 (r - 2 s)),
    # plus float32 rounding of D
    dist = np.abs(np.linalg.norm(tri - c, axis=-1) - r)
    assert dist.max() <= s * s / (8 * (r - 2 * s)) + 1e-6
    V, edges, F = _mesh_topology(tri)
    # closed and consistently oriented: every edge in exactly two triangles, opposite ways
    for k, uses in edges.items():
        assert len(uses) == 2 and uses[0] == (uses[1][1], uses[1][0]), k
    assert V - len(edges) + F == 2
    # enclosed volume (divergence theorem), outward normals give a positive volume
    vol = np.einsum("ij,ij->i", tri[:, 0] - c, np.cross(tri[:, 1] - c, tri[:, 2] - c)).sum() / 6.0
    assert abs(vol - 4.0 / 3.0 * math.pi * r ** 3) < 0.01 * 4.0 / 3.0 * math.pi * r ** 3
    # the cube ids name the cube whose corners bracket each vertex
    lo = cube[:, None, :3] * s
    assert np.all(tri >= lo - 1e-12) and np.all(tri <= lo + s + 1e-12)
