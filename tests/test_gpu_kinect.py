"""Kinect-scale workload (640x480, 1 cm voxels, 4 cm truncation, 2^20 buckets; 600
frames fused 10 per keyframe into 60 keyframes, integrated at drifted poses, one pose
update re-integrating all 60), in the launch configuration the benchmark times.

* oracle parity at full resolution on the first 6 keyframes (keyframe depth = the
  oracle's own Eq. 1 fusion, so no oracle input comes from the GPU);
* at full size (60 keyframes) properties that hold at any size: the batched update
  equals the per-keyframe path, integrating in one launch equals per-keyframe
  integration, weights are exact integers, the update is exactly undone by the
  reverse update."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import compare_volumes, flag_bound, _keys
from paper_1709_03763_b300 import Volume, fuse_keyframes, synthetic

pytestmark = pytest.mark.gpu
KAPPA = 10


@pytest.fixture(scope="module")
def kin():
    w = synthetic.workload_kinect(device="cuda")
    nf = 600
    Zg, Wg = fuse_keyframes(w.frames_depth, w.frame_poses, [f // KAPPA for f in range(nf)], w.frame_poses[::KAPPA],
                            w.intr)
    return w, Zg, Wg


def _vol(w, colour="rgba8", max_blocks=1 << 21):
    return Volume(w.voxel_size, w.trunc, w.n_buckets, colour=colour, max_blocks=max_blocks, max_keyframes=64,
                  max_blocks_per_keyframe=1 << 17, max_batch=64)


def _by_key(e):
    order = np.argsort(_keys(e["coords"].cpu().numpy()))
    idx = torch.from_numpy(order).to(e["coords"].device)
    return {k: v[idx] for k, v in e.items()}


def test_fusion_parity_full_resolution(kin):
    w, Zg, Wg = kin
    it = w.intr.as_tuple()
    frames = w.frames_depth[:2 * KAPPA].cpu()
    for k in range(2):
        s = k * KAPPA
        Zo, Wo, fl = oracle.fuse(frames[s:s + KAPPA], w.frame_poses[s:s + KAPPA], w.frame_poses[s], it)
        z, wt = Zg[k].cpu().numpy().astype(np.float64), Wg[k].cpu().numpy().astype(np.float64)
        good = (fl == 0) & (Wo > 0)
        assert good.sum() > 0.5 * Wo.size
        # flagged target pixels, as the oracle measures them: 2.2-2.3 %, bounded at 1.5x
        print(f"[fusion parity kinect {k}] flagged {100 * (fl != 0).mean():.2f} % of keyframe pixels")
        assert (fl != 0).mean() <= 1.5 * 0.0232
        assert np.all((wt[fl == 0] > 0) == (Wo[fl == 0] > 0))
        assert np.abs(z - Zo)[good].max() <= 1e-5
        assert (np.abs(wt - Wo)[good] * Zo[good] ** 2).max() <= 1e-5


@pytest.mark.parametrize("colour", ["f32", "rgba8"])
def test_integration_and_update_parity_full_resolution(kin, colour):
    w, _, _ = kin
    it = w.intr.as_tuple()
    n = 6
    frames = w.frames_depth[:n * KAPPA].cpu()
    depth = []
    for k in range(n):
        s = k * KAPPA
        Zo, _, _ = oracle.fuse(frames[s:s + KAPPA], w.frame_poses[s:s + KAPPA], w.frame_poses[s], it)
        depth.append(Zo.astype(np.float32))
    depth = np.stack(depth)
    rgba = w.kf_rgba[:n].contiguous()
    D, C = torch.from_numpy(depth).cuda(), rgba.cuda()
    V = _vol(w, colour, max_blocks=1 << 18)
    O = oracle.Volume(w.voxel_size, w.trunc, rgba8=(colour == "rgba8"))
    V.integrate_many(list(range(n)), D, C, w.kf_poses[:n], w.intr)
    for k in range(n):
        O.integrate(k, depth[k], rgba[k].cpu(), it, w.kf_poses[k])
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("kinect6"), colour=colour,
                    c_tol=0.5 if colour == "f32" else 2.0, label=f"kinect6 integrate {colour}")
    ids = list(range(n))
    V.reintegrate_batch(ids, D, C, w.kf_poses[:n], w.new_poses[:n], w.intr)
    O.reintegrate_batch(ids, depth, rgba.cpu(), w.kf_poses[:n], w.new_poses[:n], it)
    V.check()
    r = compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("kinect6"), colour=colour,
                        c_tol=0.5 if colour == "f32" else 3.0, label=f"kinect6 update {colour}")
    assert r["observed"] > 1_000_000


def test_full_size_batched_equals_plain(kin):
    """60 keyframes: one batched update == 120 per-keyframe calls; one-launch
    integration == 60 per-keyframe integrations."""
    w, Zg, _ = kin
    C = w.kf_rgba.contiguous()
    ids = list(range(60))
    A = _vol(w, "f32")
    B = _vol(w, "f32")
    A.integrate_many(ids, Zg, C, w.kf_poses, w.intr)
    for k in ids:
        B.integrate(k, Zg[k], C[k], w.intr, w.kf_poses[k])
    ea, eb = _by_key(A.extract()), _by_key(B.extract())
    assert torch.equal(ea["coords"], eb["coords"]) and torch.equal(ea["W"], eb["W"])
    assert (ea["D"] - eb["D"]).abs().max().item() <= 1e-5
    assert (ea["C"] - eb["C"]).abs().max().item() <= 0.5
    A.reintegrate_batch(ids, Zg, C, w.kf_poses, w.new_poses, w.intr)
    for k in ids:
        B.deintegrate(k, Zg[k], C[k], w.intr, w.kf_poses[k])
    for k in ids:
        B.integrate(k, Zg[k], C[k], w.intr, w.new_poses[k])
    A.check()
    B.check()
    ea, eb = _by_key(A.extract()), _by_key(B.extract())
    assert torch.equal(ea["coords"], eb["coords"]) and torch.equal(ea["W"], eb["W"])
    obs = eb["W"] > 0
    assert (ea["D"] - eb["D"])[obs].abs().max().item() <= 1e-5
    assert (ea["C"] - eb["C"])[obs].abs().max().item() <= 0.5
    # weights count observations exactly
    assert torch.equal(ea["W"], ea["W"].round())
    n_blocks = ea["coords"].shape[0]
    for k in (0, 30, 59):
        assert A.keyframe_blocks(k).numel() > 1000
    # the reverse update restores the integrated volume's weights
    A.reintegrate_batch(ids, Zg, C, w.new_poses, w.kf_poses, w.intr)
    R = _vol(w, "f32")
    R.integrate_many(ids, Zg, C, w.kf_poses, w.intr)
    ea, er = A.extract(), _by_key(R.extract())
    ka = _keys(ea["coords"].cpu().numpy())
    ia = {k: i for i, k in enumerate(ka.tolist())}
    I = np.array([ia[k] for k in _keys(er["coords"].cpu().numpy()).tolist()])
    assert torch.equal(ea["W"][I], er["W"])
    assert (ea["D"][I] - er["D"]).abs().max().item() <= 2e-5
    assert n_blocks >= er["coords"].shape[0]
