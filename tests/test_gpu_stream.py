"""GPU streaming sphere (Section 3 "SDF volume"; the streaming order of Section 4.3):
the resident set after a stream-out equals the oracle's partition, streaming changes
no voxel, de-integration and batched re-integration across streaming equal the
unstreamed volume and the oracle, non-resident keyframes are refused before any
launch, and a block allocated while stored is reported on stream-in."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import compare_volumes, flag_bound
from paper_1709_03763_b300 import BlockStore, SurfcorrError, Volume, _lib, synthetic

pytestmark = pytest.mark.gpu


def _by_key(ex):
    c = ex["coords"].cpu().numpy()
    order = np.lexsort(c.T[::-1])
    return (c[order], ex["D"].cpu().numpy()[order], ex["W"].cpu().numpy()[order], ex["C"].cpu().numpy()[order])


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _volume(w, colour="f32"):
    return Volume(w.voxel_size, w.trunc, w.n_buckets, max_blocks=1 << 16, colour=colour, max_keyframes=16,
                  max_batch=16)


def _camera(T):
    return np.asarray(T, np.float32)[:, 3]


def test_stream_out_partition_and_round_trip():
    w = synthetic.workload_tiny()
    V = _volume(w)
    for k in range(4):
        V.integrate(k, w.kf_depth[k].cuda(), w.kf_rgba[k].cuda(), w.intr, w.kf_poses[k])
    before = _by_key(V.extract())
    S = BlockStore(1 << 14, "f32")
    centre = _camera(w.kf_poses[0])
    radius = 1.2
    n_out = V.stream_out(S, centre, radius)
    out, marg = oracle.sphere_outside(before[0], w.voxel_size, centre, radius)
    assert 0 < n_out < len(before[0]) and len(S) == n_out
    after = _by_key(V.extract())
    resident = {tuple(c) for c in after[0]}
    for i, c in enumerate(before[0]):
        if not marg[i]:
            assert (tuple(c) in resident) == (not out[i])
    # the resident blocks keep their data exactly
    idx = {tuple(c): i for i, c in enumerate(before[0])}
    sel = np.array([idx[tuple(c)] for c in after[0]])
    _same(after[1:], (before[1][sel], before[2][sel], before[3][sel]))
    # everything back: the identical volume
    assert V.stream_in(S, centre) == n_out and len(S) == 0
    _same(_by_key(V.extract()), before)
    V.close()
    S.close()


def test_deintegration_across_streaming_equals_unstreamed_and_oracle():
    w = synthetic.workload_tiny()
    it = w.intr.as_tuple()
    V, R = _volume(w), _volume(w)
    O = oracle.Volume(w.voxel_size, w.trunc)
    for k in range(4):
        for vol in (V, R):
            vol.integrate(k, w.kf_depth[k].cuda(), w.kf_rgba[k].cuda(), w.intr, w.kf_poses[k])
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    S = BlockStore(1 << 14, "f32")
    V.stream_out(S, _camera(w.kf_poses[0]), 0.6)
    snap = _by_key(V.extract())
    # keyframe 2 now names stored blocks: refused before any launch, nothing changes
    with pytest.raises(SurfcorrError) as e:
        V.deintegrate(2, w.kf_depth[2].cuda(), w.kf_rgba[2].cuda(), w.intr, w.kf_poses[2])
    assert e.value.code == _lib.SC_ERR_NOT_RESIDENT
    _same(_by_key(V.extract()), snap)
    # stream in exactly the blocks keyframe 2 needs, de-integrate it, then the rest
    stored = len(S)
    n2 = V.stream_in_keyframes(S, [2])
    assert 0 < n2 <= stored and len(S) == stored - n2
    assert V.stream_in_keyframes(S, [2]) == 0  # nothing left to bring in for it
    for vol in (V, R):
        vol.deintegrate(2, w.kf_depth[2].cuda(), w.kf_rgba[2].cuda(), w.intr, w.kf_poses[2])
    V.stream_in(S, _camera(w.kf_poses[2]))
    O.deintegrate(2, w.kf_depth[2], w.kf_rgba[2], it, w.kf_poses[2])
    _same(_by_key(V.extract()), _by_key(R.extract()))
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny_stream"), label="stream de-integration")
    for x in (V, R, S):
        x.close()


def test_batched_reintegration_with_streaming_protocol():
    # Section 4.3: stream in the spheres around the selected keyframes' former and
    # updated poses, re-integrate them in one batch, stream back out around the camera
    w = synthetic.workload_tiny()
    it = w.intr.as_tuple()
    V, R = _volume(w), _volume(w)
    O = oracle.Volume(w.voxel_size, w.trunc)
    K = 6
    for k in range(K):
        for vol in (V, R):
            vol.integrate(k, w.kf_depth[k].cuda(), w.kf_rgba[k].cuda(), w.intr, w.kf_poses[k])
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    g = synthetic.rng(1, 77)
    new = w.kf_poses[:K].copy()
    for k in range(K):
        new[k] = synthetic.perturb_pose(w.kf_poses[k], np.radians(0.5), 0.01, g).astype(np.float32)
    S = BlockStore(1 << 14, "f32")
    cam = _camera(w.kf_poses[K - 1])
    V.stream_out(S, cam, 0.8)
    ids = [1, 2, 3]
    for k in ids:
        V.stream_in(S, _camera(w.kf_poses[k]), 5.0)
        V.stream_in(S, _camera(new[k]), 5.0)
    D = torch.stack([w.kf_depth[k] for k in ids]).cuda()
    C = torch.stack([w.kf_rgba[k] for k in ids]).cuda()
    for vol in (V, R):
        vol.reintegrate_batch(ids, D, C, w.kf_poses[ids], new[ids], w.intr)
    O.reintegrate_batch(ids, w.kf_depth[ids], w.kf_rgba[ids], w.kf_poses[ids], new[ids], it)
    V.stream_out(S, cam, 0.8)
    V.stream_in(S, cam)
    _same(_by_key(V.extract()), _by_key(R.extract()))
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny_stream"), label="stream batch")
    for x in (V, R, S):
        x.close()


def test_block_allocated_while_stored_conflicts():
    w = synthetic.workload_tiny()
    V = _volume(w, colour="rgba8")
    V.integrate(0, w.kf_depth[0].cuda(), w.kf_rgba[0].cuda(), w.intr, w.kf_poses[0])
    S = BlockStore(1 << 14)
    n = V.stream_out(S, _camera(w.kf_poses[0]), 0.0)  # everything out
    assert n == len(S) > 0 and V.info()["allocated_blocks"] == 0
    V.integrate(1, w.kf_depth[0].cuda(), w.kf_rgba[0].cuda(), w.intr, w.kf_poses[0])  # same region again
    with pytest.raises(SurfcorrError) as e:
        V.stream_in(S, _camera(w.kf_poses[0]))
    assert e.value.code == _lib.SC_ERR_CONFLICT
    assert len(S) == n  # the conflicting blocks stay stored
    V.close()
    S.close()


def test_store_capacity_and_empty_cases():
    w = synthetic.workload_tiny()
    V = _volume(w, colour="rgba8")
    V.integrate(0, w.kf_depth[0].cuda(), w.kf_rgba[0].cuda(), w.intr, w.kf_poses[0])
    n = V.info()["allocated_blocks"]
    small = BlockStore(max(1, n // 4))
    with pytest.raises(SurfcorrError) as e:  # more blocks than the store holds: nothing moves
        V.stream_out(small, _camera(w.kf_poses[0]), 0.0)
    assert e.value.code == _lib.SC_ERR_CAPACITY
    assert len(small) == 0 and V.info()["allocated_blocks"] == n
    big = BlockStore(n + 16)
    assert V.stream_out(big, _camera(w.kf_poses[0]), 1e6) == 0      # everything inside: nothing moves
    assert V.stream_in(big, _camera(w.kf_poses[0])) == 0             # empty store
    with pytest.raises(SurfcorrError):                               # colour formats must match
        V.stream_out(BlockStore(16, "f32"), _camera(w.kf_poses[0]), 0.0)
    for x in (V, small, big):
        x.close()


def test_stream_in_poses_brings_back_exactly_what_the_new_allocation_reaches():
    # Section 4.3: before re-integrating keyframes at updated poses, the blocks their
    # lists name (sc_stream_in_keyframes) and the stored blocks the updated poses'
    # allocation reaches (sc_stream_in_poses, the allocation's own walk) are brought in;
    # the batch then allocates no second copy of a stored block (streaming everything
    # back raises no conflict), equals the unstreamed volume bit for bit, and every
    # block the poses brought in is in some updated keyframe's new block list
    w = synthetic.workload_tiny()
    V, R = _volume(w), _volume(w)
    K = 6
    for k in range(K):
        for vol in (V, R):
            vol.integrate(k, w.kf_depth[k].cuda(), w.kf_rgba[k].cuda(), w.intr, w.kf_poses[k])
    g = synthetic.rng(1, 78)
    new = w.kf_poses[:K].copy()
    for k in range(K):
        new[k] = synthetic.perturb_pose(w.kf_poses[k], np.radians(2.0), 0.05, g).astype(np.float32)
    S = BlockStore(1 << 14, "f32")
    cam = _camera(w.kf_poses[K - 1])
    V.stream_out(S, cam, 0.7)
    ids = [1, 2, 3]
    D = torch.stack([w.kf_depth[k] for k in ids]).cuda()
    C = torch.stack([w.kf_rgba[k] for k in ids]).cuda()
    key = lambda c: {tuple(x) for x in c.tolist()}
    V.stream_in_keyframes(S, ids)
    mid = key(V.extract(payload=False)["coords"].cpu())
    n_pose = V.stream_in_poses(S, D, new[ids], w.intr)
    after = key(V.extract(payload=False)["coords"].cpu())
    brought = after - mid
    assert n_pose == len(brought) > 0
    assert V.stream_in_poses(S, D, new[ids], w.intr) == 0  # nothing left to bring in for them
    for vol in (V, R):
        vol.reintegrate_batch(ids, D, C, w.kf_poses[ids], new[ids], w.intr)
    ex = V.extract(payload=False)
    slot2c = dict(zip(ex["slots"].cpu().tolist(), map(tuple, ex["coords"].cpu().tolist())))
    listed = set()
    for k in ids:
        listed |= {slot2c[s] for s in V.keyframe_blocks(k).cpu().tolist()}
    assert brought <= listed
    V.stream_in(S, cam)  # everything back: raises SC_ERR_CONFLICT on a duplicated block
    assert len(S) == 0
    _same(_by_key(V.extract()), _by_key(R.extract()))
    for x in (V, R, S):
        x.close()


def test_stream_in_poses_argument_errors():
    w = synthetic.workload_tiny()
    V = _volume(w)
    S = BlockStore(64, "f32")
    d = w.kf_depth[:1].cuda()
    assert V.stream_in_poses(S, d[:0], w.kf_poses[:0], w.intr) == 0  # nothing to do
    bad = w.kf_poses[:1].copy()
    bad[0, 0, 3] = np.nan
    with pytest.raises(SurfcorrError):
        V.stream_in_poses(S, d, bad, w.intr)
    S2 = BlockStore(64, "rgba8")  # colour format of another volume kind
    with pytest.raises(SurfcorrError):
        V.stream_in_poses(S2, d, w.kf_poses[:1], w.intr)
    for x in (V, S, S2):
        x.close()
