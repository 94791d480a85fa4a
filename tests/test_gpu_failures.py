"""Failure paths: full pool, full hash table, full block list, bad arguments.  Tiny
capacities force them; every device wait is bounded, nothing traps or hangs."""
import numpy as np
import pytest
import torch

from gpu_helpers import cuda, gpu_volume
from paper_1709_03763_b300 import SurfcorrError, Volume, _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tinyg(tiny):
    return tiny, cuda(tiny.kf_depth), cuda(tiny.kf_rgba)


def test_pool_full(tinyg):
    w, D, C = tinyg
    V = gpu_volume(w, max_blocks=64)
    V.integrate(0, D[0], C[0], w.intr, w.kf_poses[0])
    assert V.status() == _lib.SC_ERR_POOL_FULL
    assert V.info()["allocated_blocks"] == 64


def test_hash_full(tinyg):
    w, D, C = tinyg
    V = Volume(w.voxel_size, w.trunc, 16, bucket_size=1, max_blocks=4096)
    V.integrate(0, D[0], C[0], w.intr, w.kf_poses[0])
    assert V.status() == _lib.SC_ERR_HASH_FULL


def test_list_full(tinyg):
    w, D, C = tinyg
    V = gpu_volume(w, max_blocks_per_keyframe=32)
    V.integrate(0, D[0], C[0], w.intr, w.kf_poses[0])
    assert V.status() == _lib.SC_ERR_LIST_FULL


def test_retry_limit_one_does_not_hang(tinyg):
    w, D, C = tinyg
    V = gpu_volume(w)
    V.set_retry_limit(1)
    for k in range(3):
        V.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
    assert V.status() in (0, _lib.SC_ERR_RETRY_LIMIT)


def test_argument_errors(tinyg):
    w, D, C = tinyg
    V = gpu_volume(w, max_keyframes=4)
    with pytest.raises(SurfcorrError) as e:
        V.integrate(4, D[0], C[0], w.intr, w.kf_poses[0])
    assert e.value.code == _lib.SC_ERR_INVALID_ARG
    V.integrate(3, D[0], C[0], w.intr, w.kf_poses[0])
    with pytest.raises(SurfcorrError) as e:
        V.integrate(3, D[0], C[0], w.intr, w.kf_poses[0])
    assert e.value.code == _lib.SC_ERR_ALREADY_INTEGRATED
    with pytest.raises(SurfcorrError) as e:
        V.deintegrate(1, D[0], C[0], w.intr, w.kf_poses[0])
    assert e.value.code == _lib.SC_ERR_NOT_INTEGRATED
    flat = D[0].flatten()
    with pytest.raises(SurfcorrError) as e:  # misaligned device pointer
        V.integrate(0, flat[1:1 + flat.numel() - 1], C[0], w.intr, w.kf_poses[0])
    bad = w.kf_poses[0].copy()
    bad[0, 3] = np.nan
    with pytest.raises(SurfcorrError):
        V.integrate(0, D[0], C[0], w.intr, bad)
    with pytest.raises(SurfcorrError):
        V.reintegrate_batch([3, 3], D[:2], C[:2], w.kf_poses[:2], w.kf_poses[:2], w.intr)
    with pytest.raises(SurfcorrError):
        Volume(0.01, 0.04, 1000)  # bucket count not a power of two


def test_extract_capacity_reports_true_count(tinyg):
    w, D, C = tinyg
    V = gpu_volume(w)
    V.integrate(0, D[0], C[0], w.intr, w.kf_poses[0])
    n = V.info()["allocated_blocks"]
    with pytest.raises(SurfcorrError) as e:
        V.extract(payload=True, capacity=n // 2)
    assert e.value.code == _lib.SC_ERR_CAPACITY
    full = V.extract()
    assert full["coords"].shape[0] == n


def test_batched_calls_report_device_errors_through_the_status(tinyg):
    # batched integration and pose updates launch without synchronising: a full pool
    # does not fail the call, it sets the sticky status that sc_get_status reads
    w, D, C = tinyg
    V = gpu_volume(w, max_blocks=64)
    ids = [0, 1]
    V.integrate_many(ids, D[ids], C[ids], w.kf_poses[ids], w.intr)
    assert V.status() == _lib.SC_ERR_POOL_FULL
    assert V.status() == 0  # read and cleared
    # back-to-back batched calls alternate their staging tables: a third call reuses the
    # first one's, after that launch has read it
    W2 = gpu_volume(w)
    for k in range(3):
        W2.integrate_many([k], D[k:k + 1], C[k:k + 1], w.kf_poses[k:k + 1], w.intr)
    W2.check()
    O = gpu_volume(w)
    for k in range(3):
        O.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
    a, b = W2.extract(), O.extract()
    assert a["coords"].shape == b["coords"].shape
