"""Batched re-integration (Section 4.3) on the GPU: one graph launch per pose update,
compared with the oracle's sequential semantics (de-integrate every item at its former
pose, then integrate every item at its updated pose)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import compare_volumes, cuda, flag_bound, gpu_volume, oracle_volume, _keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tinyg(tiny):
    return tiny, cuda(tiny.kf_depth), cuda(tiny.kf_rgba)


def _by_key(e):
    """Extract sorted by block key (extraction order is unspecified)."""
    order = np.argsort(_keys(e["coords"].cpu().numpy()))
    idx = torch.from_numpy(order).to(e["coords"].device)
    return {k: v[idx] for k, v in e.items()}


def _integrate_all(V, O, w, D, C):
    it = w.intr.as_tuple()
    for k in range(10):
        V.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
        if O is not None:
            O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])


@pytest.mark.parametrize("colour", ["f32", "rgba8"])
def test_batch_matches_sequential_oracle(tinyg, colour):
    w, D, C = tinyg
    ids = [int(i) for i in w.update_ids]
    V = gpu_volume(w, colour=colour)
    O = oracle_volume(w, rgba8=(colour == "rgba8"))
    _integrate_all(V, O, w, D, C)
    V.reintegrate_batch(ids, D[ids], C[ids], w.kf_poses[ids], w.new_poses[ids], w.intr)
    O.reintegrate_batch(ids, w.kf_depth[ids], w.kf_rgba[ids], w.kf_poses[ids], w.new_poses[ids], w.intr.as_tuple())
    # RGBA8: the batch rounds colour once per voxel, the sequential reference after every
    # keyframe operation; each rounding moves a channel by at most half a level
    r = compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny"), colour=colour,
                        c_tol=0.5 if colour == "f32" else 2.0, label=f"tiny batch {colour}")
    # the new block lists equal the updated poses' allocation sets
    for k in ids:
        assert V.keyframe_blocks(k).numel() > 0


def test_batch_block_lists_equal_plain_integration(tinyg):
    w, D, C = tinyg
    ids = [int(i) for i in w.update_ids]
    A = gpu_volume(w)
    _integrate_all(A, None, w, D, C)
    A.reintegrate_batch(ids, D[ids], C[ids], w.kf_poses[ids], w.new_poses[ids], w.intr)
    B = gpu_volume(w)
    for k in range(10):
        B.integrate(k, D[k], C[k], w.intr, w.new_poses[k] if k in ids else w.kf_poses[k])
    ea, eb = A.extract(payload=False), B.extract(payload=False)
    sa = dict(zip(ea["slots"].cpu().tolist(), _keys(ea["coords"].cpu().numpy()).tolist()))
    sb = dict(zip(eb["slots"].cpu().tolist(), _keys(eb["coords"].cpu().numpy()).tolist()))
    for k in range(10):
        la = sorted(sa[s] for s in A.keyframe_blocks(k).cpu().tolist())
        lb = sorted(sb[s] for s in B.keyframe_blocks(k).cpu().tolist())
        assert la == lb, k


def test_batch_all_keyframes_and_identity_update(tinyg):
    """Re-integrating every keyframe at its own pose leaves the volume unchanged (up to
    float rounding of the net change); then a full update matches the oracle."""
    w, D, C = tinyg
    ids = list(range(10))
    V = gpu_volume(w)
    _integrate_all(V, None, w, D, C)
    e0 = _by_key(V.extract())
    V.reintegrate_batch(ids, D, C, w.kf_poses, w.kf_poses, w.intr)
    e1 = _by_key(V.extract())
    assert torch.equal(e0["coords"], e1["coords"]) and torch.equal(e0["W"], e1["W"])
    assert (e0["D"] - e1["D"]).abs().max().item() < 1e-6
    O = oracle_volume(w)
    _integrate_all(gpu_volume(w), O, w, D, C)
    new = w.kf_poses.copy()
    new[w.update_ids] = w.new_poses[w.update_ids]
    V.reintegrate_batch(ids, D, C, w.kf_poses, new, w.intr)
    O.reintegrate_batch(ids, w.kf_depth, w.kf_rgba, w.kf_poses, new, w.intr.as_tuple())
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny"), label="tiny full update")


def test_batch_then_reverse_batch_restores(tinyg):
    w, D, C = tinyg
    ids = [int(i) for i in w.update_ids]
    V = gpu_volume(w)
    _integrate_all(V, None, w, D, C)
    e0 = V.extract()
    V.reintegrate_batch(ids, D[ids], C[ids], w.kf_poses[ids], w.new_poses[ids], w.intr)
    V.reintegrate_batch(ids, D[ids], C[ids], w.new_poses[ids], w.kf_poses[ids], w.intr)
    e1 = V.extract()
    k0, k1 = _keys(e0["coords"].cpu().numpy()), _keys(e1["coords"].cpu().numpy())
    i1 = {k: i for i, k in enumerate(k1.tolist())}
    I1 = np.array([i1[k] for k in k0.tolist()])
    assert torch.equal(e0["W"], e1["W"][I1])
    assert (e0["D"] - e1["D"][I1]).abs().max().item() < 2e-6


def test_autotune_leaves_volume_unchanged(tinyg):
    w, D, C = tinyg
    ids = [int(i) for i in w.update_ids]
    V = gpu_volume(w)
    _integrate_all(V, None, w, D, C)
    e0 = _by_key(V.extract())
    cfg, ms = V.autotune_batch(ids, D[ids], C[ids], w.kf_poses[ids], w.new_poses[ids], w.intr)
    assert ms > 0 and cfg["warps_per_cta"] in (4, 8)
    e1 = _by_key(V.extract())
    assert torch.equal(e0["coords"], e1["coords"]) and torch.equal(e0["W"], e1["W"]) and torch.equal(e0["D"], e1["D"])
    # and the tuned configuration gives the same result as the default one
    V.reintegrate_batch(ids, D[ids], C[ids], w.kf_poses[ids], w.new_poses[ids], w.intr)
    B = gpu_volume(w)
    _integrate_all(B, None, w, D, C)
    B.reintegrate_batch(ids, D[ids], C[ids], w.kf_poses[ids], w.new_poses[ids], w.intr)
    ea, eb = V.extract(), B.extract()
    ka, kb = _keys(ea["coords"].cpu().numpy()), _keys(eb["coords"].cpu().numpy())
    ib = {k: i for i, k in enumerate(kb.tolist())}
    Ib = np.array([ib[k] for k in ka.tolist()])
    assert torch.equal(ea["W"], eb["W"][Ib])
    assert torch.equal(ea["D"], eb["D"][Ib])  # deterministic per-voxel summation order
