"""Oracle pin for the streaming sphere's resident set (Section 3 "SDF volume"): block
centres at known distances."""
import math

import numpy as np

import oracle


def test_blocks_around_the_centre():
    s = 0.01
    # block b's centre is at voxel 8 b + 3.5; the 8 blocks around voxel -0.5 have their
    # centres 4 voxels away on every axis: 4 sqrt(3) s
    coords = np.array([[x, y, z] for x in (-1, 0) for y in (-1, 0) for z in (-1, 0)], np.int32)
    sf = float(np.float32(s))
    c = np.array([-0.5 * sf] * 3)
    d = 4 * math.sqrt(3) * sf
    out, marg = oracle.sphere_outside(coords, s, c, d * 1.001)
    assert not out.any() and not marg.any()
    out, _ = oracle.sphere_outside(coords, s, c, d * 0.999)
    assert out.all()
    # a line of blocks along x seen from the axis: block b's centre is (8 b + 3.5) s away
    coords = np.array([[b, 0, 0] for b in range(10)], np.int32)
    c = np.array([0.0, 3.5 * sf, 3.5 * sf])
    out, _ = oracle.sphere_outside(coords, s, c, (8 * 3 + 4.0) * sf)
    assert list(np.nonzero(~out)[0]) == [0, 1, 2, 3]
