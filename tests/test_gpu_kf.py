"""GPU overlap counts and KF_OVRLP keyframe grouping (Section 4.2) against the oracle:
Kinect-scale noisy frames, the closed-form overlap of sideways views of a plane, and
edge cases (no valid pixel, a single frame, argument errors)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1709_03763_b300 import KF_OVRLP, SurfcorrError, overlap_counts, segment_keyframes, synthetic

pytestmark = pytest.mark.gpu

INTR = (60.0, 60.0, 31.5, 23.5, 64, 48)


def test_overlap_counts_match_oracle_kinect():
    w = synthetic.workload_kinect(device="cuda", render_frames=40)
    d = w.frames_depth[:40].contiguous()
    poses = w.frame_poses[:40]
    it = w.intr.as_tuple()
    for kf in (0, 17):
        c = overlap_counts(d, poses, poses[kf], w.intr).cpu().numpy()
        for f in range(0, 40, 3):
            valid, inside, marg = oracle.overlap(d[f].cpu(), poses[f], poses[kf], it)
            assert c[f, 0] == valid
            assert abs(int(c[f, 1]) - inside) <= marg
        assert c[kf, 1] == c[kf, 0]  # a frame overlaps itself completely


def test_overlap_counts_closed_form_plane():
    fx, fy, cx, cy, W, H = INTR
    z0 = 2.0
    poses = []
    for t in (0.0, 0.031, 0.25, 1.9, 2.5):
        T = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
        T[0, 3] = t
        poses.append(T)
    d = torch.full((len(poses), H, W), z0, dtype=torch.float32, device="cuda")
    c = overlap_counts(d, poses, poses[0], INTR).cpu().numpy()
    for i, T in enumerate(poses):
        s = fx * float(T[0, 3]) / z0
        assert c[i, 0] == W * H
        assert c[i, 1] == H * max(0, min(W, math.ceil(W - s - 0.5)))


@pytest.mark.parametrize("thr", [0.98, 0.95, 0.85])
def test_kf_ovrlp_grouping_matches_oracle(thr):
    n = 200
    w = synthetic.workload_kinect(device="cuda", render_frames=n)
    d = w.frames_depth[:n].contiguous()
    poses = w.frame_poses[:n]
    fk, g = segment_keyframes(KF_OVRLP, (thr,), poses, w.intr, d)
    fo, flag, go = oracle.segment(oracle.KF_OVRLP, (thr,), poses, w.intr.as_tuple(), d.cpu())
    # identical up to the first decision the oracle flags as marginal
    stop = int(np.argmax(flag)) if flag.any() else n
    assert np.array_equal(fk[:stop], fo[:stop])
    if not flag.any():
        assert g == go
    assert g >= 2 or thr < 0.9


def test_kf_ovrlp_edge_cases():
    fx, fy, cx, cy, W, H = INTR
    T = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    d = torch.full((4, H, W), 2.0, dtype=torch.float32, device="cuda")
    d[2] = 0.0                                # no valid pixel: ratio 0 -> a new keyframe
    fk, g = segment_keyframes(KF_OVRLP, (0.5,), [T] * 4, INTR, d)
    assert list(fk) == [0, 0, 1, 1] and g == 2
    fk, g = segment_keyframes(KF_OVRLP, (0.5,), [T], INTR, d[:1])
    assert list(fk) == [0] and g == 1
    with pytest.raises(SurfcorrError):      # threshold outside [0, 1]
        segment_keyframes(KF_OVRLP, (1.5,), [T] * 4, INTR, d)
    with pytest.raises(SurfcorrError):      # KF_OVRLP needs the depth frames
        segment_keyframes(KF_OVRLP, (0.5,), [T] * 4, INTR, None)


def test_overlap_counts_ragged_width_matches_oracle():
    # width 53: the one-pixel-per-thread kernel; a tilted plane with holes, frames
    # translated and yawed against the keyframe
    intr = (45.0, 45.0, 26.3, 18.1, 53, 37)
    W, H = 53, 37
    g = np.random.default_rng(11)
    d = np.full((5, H, W), 1.6, np.float32) + np.linspace(0.0, 0.4, W, dtype=np.float32)[None, None, :]
    d[g.random(d.shape) < 0.1] = 0.0
    poses = []
    for i in range(5):
        a = math.radians(2.0 * i)
        T = np.zeros((3, 4), np.float32)
        T[:, :3] = [[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]]
        T[0, 3] = 0.05 * i
        poses.append(T)
    c = overlap_counts(torch.from_numpy(d).cuda(), poses, poses[1], intr).cpu().numpy()
    for f in range(5):
        valid, inside, marg = oracle.overlap(torch.from_numpy(d[f]), poses[f], poses[1], intr)
        assert c[f, 0] == valid
        assert abs(int(c[f, 1]) - inside) <= marg
    assert c[1, 1] == c[1, 0]


def test_kf_ovrlp_grouping_ragged_width_matches_oracle():
    # width 53: the grouping graph's one-pixel-per-thread overlap step; frames sliding
    # sideways so that the overlap falls below the threshold every few frames, after
    # a grouping of another image size (the per-device graph is rebuilt)
    intr = (45.0, 45.0, 26.3, 18.1, 53, 37)
    W, H = 53, 37
    g = np.random.default_rng(12)
    n = 40
    d = np.full((n, H, W), 1.6, np.float32) + np.linspace(0.0, 0.4, W, dtype=np.float32)[None, None, :]
    d[g.random(d.shape) < 0.1] = 0.0
    poses = []
    for i in range(n):
        T = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
        T[0, 3] = np.float32(0.05 * i)
        poses.append(T)
    dt = torch.from_numpy(d).cuda()
    for thr in (0.9, 0.7):
        fk, gk = segment_keyframes(KF_OVRLP, (thr,), poses, intr, dt)
        fo, flag, go = oracle.segment(oracle.KF_OVRLP, (thr,), poses, intr, torch.from_numpy(d))
        stop = int(np.argmax(flag)) if flag.any() else n
        assert np.array_equal(fk[:stop], fo[:stop])
        if not flag.any():
            assert gk == go
        assert gk >= 3
