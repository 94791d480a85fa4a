"""Checkpoint / resume: a volume saved (blocks + keyframe block lists as coordinates)
and loaded into a fresh volume holds identical voxels, and its restored keyframes
de-integrate and re-integrate exactly as in the original volume."""
import numpy as np
import pytest
import torch

from paper_1709_03763_b300 import SurfcorrError, Volume, _lib, synthetic

pytestmark = pytest.mark.gpu


def _by_key(ex):
    c = ex["coords"].cpu().numpy()
    o = np.lexsort(c.T[::-1])
    return c[o], ex["D"].cpu().numpy()[o], ex["W"].cpu().numpy()[o], ex["C"].cpu().numpy()[o]


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("colour", ["f32", "rgba8"])
def test_save_load_then_deintegrate_and_reintegrate(tmp_path, colour):
    w = synthetic.workload_tiny()
    mk = lambda: Volume(w.voxel_size, w.trunc, w.n_buckets, max_blocks=1 << 16, colour=colour, max_keyframes=16,
                        max_batch=16)
    A = mk()
    D = [w.kf_depth[k].cuda() for k in range(4)]
    C = [w.kf_rgba[k].cuda() for k in range(4)]
    for k in range(4):
        A.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
    path = str(tmp_path / "vol.npz")
    A.save(path, keyframes=range(4))
    B = mk()
    assert B.load(path) == [0, 1, 2, 3]
    _same(_by_key(B.extract()), _by_key(A.extract()))
    for vol in (A, B):
        vol.deintegrate(2, D[2], C[2], w.intr, w.kf_poses[2])
    _same(_by_key(B.extract()), _by_key(A.extract()))
    new = w.kf_poses[:4].copy()
    new[1] = w.new_poses[1]
    ids = [1, 3]
    for vol in (A, B):
        vol.reintegrate_batch(ids, torch.stack([D[i] for i in ids]), torch.stack([C[i] for i in ids]),
                              w.kf_poses[ids], new[ids], w.intr)
    _same(_by_key(B.extract()), _by_key(A.extract()))
    A.close()
    B.close()


def test_restore_list_with_a_missing_block():
    w = synthetic.workload_tiny()
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, max_blocks=1 << 16, max_keyframes=16)
    V.integrate(0, w.kf_depth[0].cuda(), w.kf_rgba[0].cuda(), w.intr, w.kf_poses[0])
    coords = torch.tensor([[10 ** 5, 0, 0]], dtype=torch.int32, device="cuda")  # no such block
    with pytest.raises(SurfcorrError) as e:
        V.set_keyframe_blocks(5, coords)
    assert e.value.code == _lib.SC_ERR_INVALID_ARG
    with pytest.raises(SurfcorrError) as e:      # the keyframe stayed not integrated
        V.deintegrate(5, w.kf_depth[0].cuda(), w.kf_rgba[0].cuda(), w.intr, w.kf_poses[0])
    assert e.value.code in (_lib.SC_ERR_NOT_INTEGRATED, _lib.SC_ERR_INVALID_ARG)
    with pytest.raises(SurfcorrError) as e:      # an integrated keyframe cannot be overwritten
        V.set_keyframe_blocks(0, coords)
    assert e.value.code == _lib.SC_ERR_ALREADY_INTEGRATED
    V.close()
