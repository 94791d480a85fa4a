"""Differentiation at Kinect scale and the batched forward + backward.

* gradients of the SDF loss w.r.t. keyframe se(3) poses and depth pixels vs the FP64
  oracle at 640x480 (first 6 keyframes, oracle-fused depth), within 1e-4 of the
  gradient scale plus the oracle's budget for marginal decisions;
* 256 keyframes of the batching scene: one forward (integration in one launch) and one
  adjoint launch for all 256 equal 256 per-keyframe integrations + the adjoint run per
  keyframe."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_03763_b300 import Volume, synthetic

pytestmark = pytest.mark.gpu
KAPPA = 10


def test_gradients_full_resolution():
    w = synthetic.workload_kinect(device="cuda", render_frames=6 * KAPPA)
    it = w.intr.as_tuple()
    n = 6
    frames = w.frames_depth[:n * KAPPA].cpu()
    depth = np.stack([oracle.fuse(frames[k * KAPPA:(k + 1) * KAPPA], w.frame_poses[k * KAPPA:(k + 1) * KAPPA],
                                  w.frame_poses[k * KAPPA], it)[0].astype(np.float32) for k in range(n)])
    rgba = w.kf_rgba[:n].contiguous()
    D = torch.from_numpy(depth).cuda()
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, colour="f32", max_blocks=1 << 18, max_keyframes=8)
    O = oracle.Volume(w.voxel_size, w.trunc)
    V.integrate_many(list(range(n)), D, rgba.cuda(), w.kf_poses[:n], w.intr)
    for k in range(n):
        O.integrate(k, depth[k], rgba[k].cpu(), it, w.kf_poses[k])
    pts = synthetic.surface_points(w.scene, 200_000, 4, lo=np.array([1.5, 0.0, 0.0]),
                                   hi=np.array([6.0, 6.0, 3.0])).astype(np.float32).astype(np.float64)
    _, _, pf = O.loss(pts)
    pts = pts[pf == 0]
    out, gD = V.sdf_loss(torch.tensor(pts, dtype=torch.float32).cuda(), 0.1)
    Lo, Po, _ = O.loss(pts, 0.1)
    assert out[1].item() == Po and Po > 1000
    assert abs(out[0].item() - Lo) <= 1e-4 * abs(Lo)
    ids = list(range(n))
    gx, gd = V.sdf_adjoint(ids, [D[k] for k in ids], w.kf_poses[:n], w.intr, gD)
    ox, od, ex, ed = O.grad(ids, depth, w.kf_poses[:n], it, pts, 0.1, with_budget=True)
    gx, gd = gx.cpu().numpy(), gd.cpu().numpy()
    scale = np.abs(ox).max()
    for k in ids:
        assert np.all(np.abs(gx[k] - ox[k]) <= 1e-4 * scale + 1.01 * ex[k]), (k, gx[k], ox[k], ex[k])
        assert np.all(np.abs(gd[k] - od[k]) <= 1e-4 * np.abs(od).max() + 1.01 * ed[k]), k


def test_batched_forward_backward_256_keyframes():
    w = synthetic.workload_batching(device="cuda", n_keyframes=256, n_updates=1)
    K = 256
    D, C = w.kf_depth, w.kf_rgba
    pts = torch.tensor(synthetic.surface_points(w.scene, 1_000_000, 5), dtype=torch.float32).cuda()
    mk = lambda: Volume(w.voxel_size, w.trunc, w.n_buckets, colour="rgba8", max_blocks=1 << 21,
                        max_keyframes=K, max_blocks_per_keyframe=1 << 16, max_batch=256)
    A, B = mk(), mk()
    ids = list(range(K))
    A.integrate_many(ids, D, C, w.kf_poses, w.intr)          # batched forward (one graph launch)
    for k in ids:
        B.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])    # 256 plain integrations
    oa, ga = A.sdf_loss(pts, 0.1)
    ob, gb = B.sdf_loss(pts, 0.1)
    assert oa[1].item() == ob[1].item() and oa[1].item() > 10000
    assert abs(oa[0].item() - ob[0].item()) <= 1e-5 * abs(ob[0].item())
    gxa, gda = A.sdf_adjoint(ids, D, w.kf_poses, w.intr, ga)  # one launch for all 256
    gxa = gxa.cpu().numpy()
    scale = np.abs(gxa).max()
    assert scale > 0
    # the same volume, one adjoint call per keyframe: only the double accumulation
    # order differs
    per = np.concatenate([A.sdf_adjoint([k], D[k:k + 1], w.kf_poses[k:k + 1], w.intr, ga, with_depth=False)[0]
                          .cpu().numpy() for k in ids])
    assert np.abs(gxa - per).max() <= 1e-9 * scale
    # against the 256 plain integrations + per-keyframe backward: the forward states
    # differ by float rounding of the running averages, which the loss amplifies
    gxb = np.concatenate([B.sdf_adjoint([k], D[k:k + 1], w.kf_poses[k:k + 1], w.intr, gb, with_depth=False)[0]
                          .cpu().numpy() for k in ids])
    assert np.abs(gxa - gxb).max() <= 1e-3 * scale
