"""The adjoint as a vector-Jacobian product on identical inputs (extension; no counterpart
in the paper): the GPU volume is the oracle's own volume imported block by block (W
exact, D rounded to float32), every keyframe's block list is the oracle's A(k, T)
(sc_set_keyframe_blocks), and both sides contract the same seeded cotangent dL/dD.  The
cotangent is zero on every voxel where the oracle took a decision within its margin
(pixel rounding, band edge, clamp kink, camera plane, marginal allocation), so the two
sides take the same decisions on every contributing sample and the oracle's error
budget is exactly zero: each keyframe's pose gradient must match the oracle's to 1e-4
of its own largest component, and central differences of the oracle's frozen-decision
functional likewise; depth-pixel gradients match per pixel."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import _keys
from paper_1709_03763_b300 import Volume, synthetic

pytestmark = pytest.mark.gpu
REL = 1e-4


def _setup(w, depth, rgba, poses, ids, seed):
    it = w.intr.as_tuple()
    O = oracle.Volume(w.voxel_size, w.trunc)
    for i, k in enumerate(ids):
        O.integrate(k, depth[i], rgba[i], it, poses[i])
    ex = O.export()
    kink = O.kink_flags()
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, colour="f32", max_blocks=max(1 << 16, 2 * len(ex.coords)),
               max_keyframes=max(ids) + 1, max_blocks_per_keyframe=1 << 17)
    coords = torch.from_numpy(ex.coords).cuda()
    V.import_blocks(coords, torch.from_numpy(ex.D.astype(np.float32)).cuda(),
                    torch.from_numpy(ex.W.astype(np.float32)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(ex.C.transpose(0, 2, 1)).astype(np.float32)).cuda())
    for k in ids:
        c, m = O.touched(k)
        V.set_keyframe_blocks(k, torch.from_numpy(np.ascontiguousarray(c[m != 2])).cuda())
    # the seeded cotangent (float32 values, the same on both sides), zero where a decision
    # was within its margin and on unobserved voxels
    g = np.random.default_rng(seed).standard_normal(ex.W.shape).astype(np.float32)
    robust = (ex.W > 0) & (ex.vflag == 0) & (kink == 0) & (ex.bflag[:, None] == 0)
    g = np.where(robust, g, np.float32(0))
    # the GPU's dL/dD is indexed by pool slot
    e = V.extract(payload=False)
    slot_of = dict(zip(_keys(e["coords"].cpu().numpy()).tolist(), e["slots"].cpu().numpy().tolist()))
    slots = np.array([slot_of[k] for k in _keys(ex.coords).tolist()])
    gD = V.grad_buffer()
    gD[torch.from_numpy(slots).cuda()] = torch.from_numpy(g).cuda()
    return O, V, ex.coords, g.astype(np.float64), gD, robust


def _check(w, O, V, ids, depth, poses, gc, gv, gD, fd_ids):
    it = w.intr.as_tuple()
    D = torch.from_numpy(np.ascontiguousarray(depth)).cuda()
    gx, gd = V.sdf_adjoint(ids, [D[i] for i in range(len(ids))], poses, w.intr, gD)
    gx, gd = gx.cpu().numpy(), gd.cpu().numpy()
    ox, od, ex, ed = O.adjoint(ids, depth, poses, it, gc, gv)
    assert not ex.any() and not ed.any()  # no contributing sample is marginal
    for i, k in enumerate(ids):
        s = np.abs(ox[i]).max()
        assert s > 0
        assert np.abs(gx[i] - ox[i]).max() <= REL * s, (k, gx[i], ox[i])
        sd = np.abs(od[i]).max()
        assert np.abs(gd[i] - od[i]).max() <= REL * sd, k
    eps = 1e-4
    for i in fd_ids:
        k = ids[i]
        fd = np.zeros(6)
        for j in range(6):
            e = np.zeros(6)
            e[j] = eps
            fd[j] = (O.adjoint_functional(k, depth[i], poses[i], it, e, gc, gv)
                     - O.adjoint_functional(k, depth[i], poses[i], it, -e, gc, gv)) / (2 * eps)
        assert np.abs(gx[i] - fd).max() <= REL * np.abs(fd).max(), (k, gx[i], fd)
    return gx, ox


def test_adjoint_vjp_tiny_room(tiny):
    w = tiny
    ids = list(range(10))
    O, V, gc, gv, gD, robust = _setup(w, w.kf_depth, w.kf_rgba, w.kf_poses, ids, 11)
    assert robust.sum() > 0.95 * (O.export().W > 0).sum()
    _check(w, O, V, ids, np.asarray(w.kf_depth), w.kf_poses, gc, gv, gD, fd_ids=[0, 3, 7])
    V.close()


def test_adjoint_vjp_kinect_scale():
    """640 x 480, 1 cm voxels: 6 keyframes fused by the oracle's own Eq. 1."""
    w = synthetic.workload_kinect(device="cpu", render_frames=60)
    it = w.intr.as_tuple()
    frames = w.frames_depth[:60].cpu()
    depth = np.stack([oracle.fuse(frames[k * 10:(k + 1) * 10], w.frame_poses[k * 10:(k + 1) * 10],
                                  w.frame_poses[k * 10], it)[0].astype(np.float32) for k in range(6)])
    rgba = w.kf_rgba[:6].contiguous().cpu()
    ids = list(range(6))
    O, V, gc, gv, gD, robust = _setup(w, depth, rgba, w.kf_poses[:6], ids, 12)
    _check(w, O, V, ids, depth, w.kf_poses[:6], gc, gv, gD, fd_ids=[0, 5])
    V.close()
