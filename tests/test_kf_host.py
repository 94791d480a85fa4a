"""Keyframe strategies on the host (KF_CONST, KF_DIST need no GPU): the library's
grouping equals the oracle's on seeded trajectories."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_03763_b300 import KF_CONST, KF_DIST, SurfcorrError, segment_keyframes, synthetic


def _trajectory(n, seed):
    g = np.random.default_rng(seed)
    T = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    out = [T]
    for _ in range(n - 1):
        T = synthetic.perturb_pose(T, math.radians(g.uniform(0.1, 1.5)), g.uniform(0.002, 0.02), g)
        out.append(T.astype(np.float32))
    return np.stack(out)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_kf_dist_equals_oracle(seed):
    poses = _trajectory(300, seed)
    for thr_t, thr_r in [(0.05, math.radians(3.0)), (0.2, math.radians(10.0)), (0.01, 1.0)]:
        fk, g = segment_keyframes(KF_DIST, (thr_t, thr_r), poses)
        fo, flag, go = oracle.segment(oracle.KF_DIST, (thr_t, thr_r), poses)
        assert not flag.any()
        assert np.array_equal(fk, fo) and g == go


def test_kf_const_and_kinect_trajectory():
    poses = synthetic.kinect_trajectory(600).astype(np.float32)
    fk, g = segment_keyframes(KF_CONST, (10,), poses)
    assert np.array_equal(fk, np.arange(600) // 10) and g == 60
    fk, g = segment_keyframes(KF_DIST, (0.1, math.radians(5.0)), poses)
    fo, _, go = oracle.segment(oracle.KF_DIST, (0.1, math.radians(5.0)), poses)
    assert np.array_equal(fk, fo) and 5 < g == go < 600


def test_invalid_strategy_arguments():
    poses = _trajectory(5, 0)
    with pytest.raises(SurfcorrError):
        segment_keyframes(7, (1.0,), poses)
    with pytest.raises(SurfcorrError):
        segment_keyframes(KF_CONST, (0,), poses)
    assert segment_keyframes(KF_CONST, (3,), poses[:0])[1] == 0
