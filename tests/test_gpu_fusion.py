"""GPU keyframe depth fusion (Eq. 1) against the oracle on Kinect-scale frames."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_03763_b300 import fuse_frames_into_keyframe, synthetic

pytestmark = pytest.mark.gpu


def _frames():
    scene, _ = synthetic.scene_kinect()
    poses = synthetic.kinect_trajectory(600)[100:110].astype(np.float32)
    d, c = synthetic.render(scene, synthetic.KINECT, poses)
    d = synthetic.add_sensor_noise(d, 2, first_frame=100)
    return d, poses


def test_fusion_matches_oracle():
    d, poses = _frames()
    Zg, Wg = fuse_frames_into_keyframe(d.cuda(), poses, poses[0], synthetic.KINECT, disc_rel=0.1)
    Zo, Wo, fl = oracle.fuse(d, poses, poses[0], synthetic.KINECT.as_tuple(), disc_rel=0.1)
    Zg, Wg = Zg.cpu().numpy().astype(np.float64), Wg.cpu().numpy().astype(np.float64)
    good = fl == 0
    # target pixels a marginal source may land on (the oracle flags x* and the pixel
    # across the tie): 3.0 % for these 9 warped frames, bounded at 1.5x
    print(f"[fusion parity] flagged {100 * (1 - good.mean()):.2f} % of keyframe pixels")
    assert 1 - good.mean() <= 1.5 * 0.0301
    cov = good & (Wo > 0)
    assert cov.sum() > 0.5 * Wo.size
    assert np.all((Wg[good] > 0) == (Wo[good] > 0))
    assert np.abs(Zg - Zo)[cov].max() <= 1e-5
    # W* = sum cos(theta) / Z^2: compare in cos(theta) units.  At grazing angles
    # (cos(theta) ~ 1e-3) float32 depth cannot give cos(theta) to 1e-5 relative, but
    # its absolute error stays far below 1e-5.
    assert (np.abs(Wg - Wo)[cov] * Zo[cov] ** 2).max() <= 1e-5
    assert np.quantile(np.abs(Wg - Wo)[cov] / Wo[cov], 0.999) <= 1e-5


@pytest.mark.parametrize("disc_rel", [0.1, 1.5])
def test_fusion_keyframe_pose_of_no_frame(disc_rel):
    # a keyframe pose that equals no frame's pose: every frame is warped (no identity
    # frame initialises the sums); disc_rel >= 1 also checks every neighbour's validity
    d, poses = _frames()
    rng = synthetic.rng(2, 77)
    kf = synthetic.perturb_pose(poses[4], np.radians(0.3), 0.004, rng).astype(np.float32)
    Zg, Wg = fuse_frames_into_keyframe(d.cuda(), poses, kf, synthetic.KINECT, disc_rel=disc_rel)
    Zo, Wo, fl = oracle.fuse(d, poses, kf, synthetic.KINECT.as_tuple(), disc_rel=disc_rel)
    Zg, Wg = Zg.cpu().numpy().astype(np.float64), Wg.cpu().numpy().astype(np.float64)
    good = fl == 0
    # every frame warped (10 instead of 9): 3.4 % of target pixels flagged, bounded at 1.5x
    print(f"[fusion parity, no identity frame, disc_rel {disc_rel}] flagged {100 * (1 - good.mean()):.2f} %")
    assert 1 - good.mean() <= 1.5 * 0.0338
    cov = good & (Wo > 0)
    assert cov.sum() > 0.5 * Wo.size
    assert np.all((Wg[good] > 0) == (Wo[good] > 0))
    assert np.abs(Zg - Zo)[cov].max() <= 1e-5
    assert (np.abs(Wg - Wo)[cov] * Zo[cov] ** 2).max() <= 1e-5


def test_fusion_identical_frames_and_ragged_size():
    z0 = 1.37
    H, W = 37, 53
    intr = (40.0, 40.0, 26.0, 18.0, W, H)
    T = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    d = torch.full((3, H, W), z0, dtype=torch.float32)
    Zg, Wg = fuse_frames_into_keyframe(d.cuda(), [T] * 3, T, intr)
    Zg, Wg = Zg.cpu().numpy(), Wg.cpu().numpy()
    inner = np.zeros((H, W), bool)
    inner[1:-1, 1:-1] = True
    zf = float(np.float32(z0))
    assert np.abs(Zg[inner] - zf).max() < 1e-6
    assert np.abs(Wg[inner] - 3 / zf ** 2).max() < 1e-5
    assert np.all(Wg[~inner] == 0)


def test_batched_fusion_equals_per_keyframe_fusion():
    from paper_1709_03763_b300 import fuse_keyframes
    d, poses = _frames()
    dg = d.cuda()
    # two keyframes of 5 frames each
    Zb, Wb = fuse_keyframes(dg, poses, [0] * 5 + [1] * 5, [poses[0], poses[5]], synthetic.KINECT)
    for k, s in enumerate((0, 5)):
        Zk, Wk = fuse_frames_into_keyframe(dg[s:s + 5].contiguous(), poses[s:s + 5], poses[s], synthetic.KINECT)
        assert torch.allclose(Wb[k], Wk, rtol=1e-5, atol=1e-9)
        assert torch.allclose(Zb[k], Zk, rtol=1e-6, atol=1e-7)


def test_depth_from_u16_is_one_float_multiply():
    from paper_1709_03763_b300 import depth_from_u16
    g = np.random.default_rng(5)
    raw = g.integers(0, 65536, 100003).astype(np.uint16)   # ragged tail after the 8-wide body
    raw[:5] = [0, 1, 65535, 5000, 20000]
    scale = np.float32(1.0 / 5000.0)
    t = torch.from_numpy(raw.view(np.int16)).cuda()
    out = depth_from_u16(t, float(scale)).cpu().numpy()
    assert np.array_equal(out, raw.astype(np.float32) * scale)
    assert out[0] == 0.0 and abs(out[3] - 1.0) < 1e-6


def test_rgba_from_rgb_expands_with_opaque_alpha():
    from paper_1709_03763_b300 import SurfcorrError, rgba_from_rgb
    g = np.random.default_rng(6)
    for n in (0, 1, 3, 4, 7, 100003):   # empty, below one vector, ragged tail after the 4-wide body
        rgb = torch.from_numpy(g.integers(0, 256, (n, 3), dtype=np.uint8)).cuda()
        out = rgba_from_rgb(rgb).cpu().numpy()
        ref = np.concatenate([rgb.cpu().numpy(), np.full((n, 1), 255, np.uint8)], axis=1)
        assert np.array_equal(out, ref)
    img = torch.from_numpy(g.integers(0, 256, (2, 48, 64, 3), dtype=np.uint8)).cuda()
    assert np.array_equal(rgba_from_rgb(img)[..., :3].cpu().numpy(), img.cpu().numpy())
    base = torch.zeros(4 * 11, dtype=torch.uint8, device="cuda")
    with pytest.raises(SurfcorrError):   # input not 4-byte aligned: refused before any launch
        rgba_from_rgb(base[1:1 + 30].view(10, 3), out=torch.empty((10, 4), dtype=torch.uint8, device="cuda"))
