"""GPU allocation A(k, T) (Section 3 "SDF volume") on depth images built to drive every
path of the tile walk against the oracle's brute-force slab test: independent random
depths per pixel (the tile window holds few of a tile's blocks, the shared key set and
the tile's compacted key list overflow, so phase D claims block by block), and a smooth
plane whose tiles' window reference pixels are all invalid (the window is off and every
block goes through the key set).  Both the plain path (32x16 tiles) and the batched
path (32x32 tiles) must list exactly the oracle's robust blocks."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import _keys
from paper_1709_03763_b300 import Volume, synthetic

pytestmark = pytest.mark.gpu

W, H = 96, 64
INTR = (80.0, 80.0, 47.5, 31.5, W, H)
VOXEL, TRUNC = 0.01, 0.04


def _pose():
    return synthetic.look_pose(np.array([0.3, -0.2, 1.1]), 0.7, 0.25).astype(np.float32)


def _random_depth():
    g = np.random.default_rng(1709)
    d = g.uniform(0.4, 6.0, (H, W)).astype(np.float32)
    d[g.random((H, W)) < 0.05] = 0.0
    return d


def _plane_without_references():
    # a tilted plane; the window reference pixels of both tile shapes (rows TY/4 * {1,2,3}
    # of each tile, columns 8, 16, 24 of each 32-pixel tile) are invalid
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    d = (1.5 + 0.004 * u + 0.006 * v).astype(np.float32)
    for ty in (16, 32):
        for r in range(H):
            if (r % ty) in (ty // 4, ty // 2, 3 * ty // 4):
                for c in range(W):
                    if (c % 32) in (8, 16, 24):
                        d[r, c] = 0.0
    return d


def _gpu_set(V, k):
    slots = V.keyframe_blocks(k).cpu().numpy()
    ex = V.extract(payload=False)
    s2c = dict(zip(ex["slots"].cpu().numpy().tolist(), map(tuple, ex["coords"].cpu().numpy())))
    keys = _keys(np.array([s2c[s] for s in slots]))
    assert len(set(keys.tolist())) == len(slots)  # the list holds each block once
    return set(keys.tolist())


@pytest.mark.parametrize("image", ["random", "plane_no_reference"])
@pytest.mark.parametrize("path", ["plain", "batched"])
def test_allocation_paths_match_oracle(image, path):
    depth = _random_depth() if image == "random" else _plane_without_references()
    pose = _pose()
    rgba = torch.full((H, W, 4), 128, dtype=torch.uint8, device="cuda")
    V = Volume(VOXEL, TRUNC, 1 << 18, colour="rgba8", max_blocks=1 << 17, max_keyframes=4,
               max_blocks_per_keyframe=1 << 17, max_batch=8)
    dg = torch.from_numpy(depth).cuda()
    if path == "plain":
        V.integrate(0, dg, rgba, INTR, pose)
    else:
        V.integrate_many([0], [dg], [rgba], [pose], INTR)
    V.check()
    gset = _gpu_set(V, 0)
    coords, marg = oracle.allocation_set(torch.from_numpy(depth), pose, INTR, VOXEL, TRUNC)
    keys = _keys(coords)
    robust = set(keys[marg == 0].tolist())
    anyk = set(keys.tolist())
    print(f"[allocation {image} {path}] {len(gset)} blocks, oracle {len(robust)} robust of {len(anyk)}")
    assert len(robust) > (2000 if image == "random" else 50)
    assert robust <= gset, len(robust - gset)
    assert gset <= anyk, len(gset - anyk)
    V.close()
