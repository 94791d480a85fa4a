"""Texel reuse between consecutive batches (the batch packs each item's depth and colour
into a texel image per position; a position whose keyframe, image pointers and image
binding are unchanged since the previous batch is not packed again).  A batch that may
reuse its texels gives the same volume as one that packs everything; a keyframe that
was de-integrated and integrated again with new content in the same buffers is packed
again."""
import numpy as np
import pytest
import torch

from gpu_helpers import cuda, gpu_volume, _keys

pytestmark = pytest.mark.gpu


def _by_key(e):
    order = np.argsort(_keys(e["coords"].cpu().numpy()))
    return {k: v.cpu().numpy()[order] for k, v in e.items()}


def _same(a, b):
    assert np.array_equal(a["coords"], b["coords"])
    for f in ("W", "D", "C"):
        assert np.array_equal(a[f], b[f]), f


def test_reused_texels_give_the_repacked_result(tiny):
    w = tiny
    D, C = cuda(w.kf_depth), cuda(w.kf_rgba)
    ids = [0, 1, 2, 3]
    new = w.kf_poses[ids].copy()
    new[1], new[3] = w.new_poses[1], w.new_poses[3]
    # A: batched integration, then a pose update of the same items in the same positions
    # (the update may reuse every item's texels)
    A = gpu_volume(w)
    A.integrate_many(ids, D[ids], C[ids], w.kf_poses[ids], w.intr)
    A.reintegrate_batch(ids, D[ids], C[ids], w.kf_poses[ids], new, w.intr)
    A.check()
    # B: the same, but the update lists the items in another order (every position packs)
    B = gpu_volume(w)
    B.integrate_many(ids, D[ids], C[ids], w.kf_poses[ids], w.intr)
    rev = ids[::-1]
    B.reintegrate_batch(rev, D[rev], C[rev], w.kf_poses[rev], new[::-1].copy(), w.intr)
    B.check()
    a, b = _by_key(A.extract()), _by_key(B.extract())
    assert np.array_equal(a["coords"], b["coords"])
    assert np.array_equal(a["W"], b["W"])
    assert np.abs(a["D"] - b["D"]).max() <= 1e-6  # item order changes the float summation order
    assert np.abs(a["C"] - b["C"]).max() <= 1e-3


def test_new_content_in_the_same_buffers_is_packed_again(tiny):
    w = tiny
    dep = cuda(w.kf_depth[0:1]).clone()   # one keyframe's buffers, rewritten in place below
    col = cuda(w.kf_rgba[0:1]).clone()
    other_d, other_c = cuda(w.kf_depth[1:2]), cuda(w.kf_rgba[1:2])
    T0, T1 = w.kf_poses[0:1], w.kf_poses[1:2]
    new1 = w.new_poses[1:2].copy()

    def run(batched_first):
        V = gpu_volume(w)
        if batched_first:
            V.integrate_many([0], dep, col, T0, w.intr)          # packs position 0 from dep / col
        else:
            V.integrate(0, dep[0], col[0], w.intr, T0[0])
        V.deintegrate(0, dep[0], col[0], w.intr, T0[0])
        dep.copy_(other_d)                                        # new content, same pointers
        col.copy_(other_c)
        V.integrate(0, dep[0], col[0], w.intr, T1[0])             # the keyframe binds the new images
        V.reintegrate_batch([0], dep, col, T1, new1, w.intr)      # must pack them again
        V.check()
        out = _by_key(V.extract())
        dep.copy_(cuda(w.kf_depth[0:1]))                          # restore for the next run
        col.copy_(cuda(w.kf_rgba[0:1]))
        return out

    _same(run(True), run(False))
