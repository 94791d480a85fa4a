"""GPU parity of allocation, integration and de-integration with the FP64 oracle
(Section 3 "SDF volume"; Eq. 2, Section 4.3) on the tiny room workload (320x240,
10 keyframes, 2 cm voxels, 8 cm truncation)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import compare_volumes, cuda, flag_bound, gpu_volume, oracle_volume, _keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tinyg(tiny):
    return tiny, cuda(tiny.kf_depth), cuda(tiny.kf_rgba)


def test_allocation_sets_match_oracle(tinyg):
    w, D, C = tinyg
    it = w.intr.as_tuple()
    for k in range(10):
        V = gpu_volume(w)
        V.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
        V.check()
        slots = V.keyframe_blocks(k).cpu().numpy()
        ex = V.extract(payload=False)
        slot_to_coord = dict(zip(ex["slots"].cpu().numpy().tolist(), map(tuple, ex["coords"].cpu().numpy())))
        gset = set(_keys(np.array([slot_to_coord[s] for s in slots])).tolist())
        assert len(gset) == len(slots)  # the list holds each block once
        coords, marg = oracle.allocation_set(w.kf_depth[k], w.kf_poses[k], it, w.voxel_size, w.trunc)
        keys = _keys(coords)
        robust = set(keys[marg == 0].tolist())
        anyk = set(keys.tolist())
        assert robust <= gset, len(robust - gset)
        assert gset <= anyk, len(gset - anyk)
        assert len(anyk) - len(robust) <= 1e-3 * len(robust) + 2
        V.close()


@pytest.mark.parametrize("colour", ["f32", "rgba8"])
def test_integrate_all_keyframes_matches_oracle(tinyg, colour):
    w, D, C = tinyg
    it = w.intr.as_tuple()
    V = gpu_volume(w, colour=colour)
    O = oracle_volume(w, rgba8=(colour == "rgba8"))
    for k in range(10):
        V.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    V.check()
    r = compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny"), colour=colour,
                        c_tol=0.5 if colour == "f32" else 0.0, label=f"tiny integrate {colour}")
    assert r["observed"] > 100000


@pytest.mark.parametrize("colour", ["f32", "rgba8"])
def test_plain_deintegrate_reintegrate_matches_oracle(tinyg, colour):
    w, D, C = tinyg
    it = w.intr.as_tuple()
    V = gpu_volume(w, colour=colour)
    O = oracle_volume(w, rgba8=(colour == "rgba8"))
    for k in range(10):
        V.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    for k in w.update_ids:
        V.deintegrate(int(k), D[k], C[k], w.intr, w.kf_poses[k])
        O.deintegrate(int(k), w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    for k in w.update_ids:
        V.integrate(int(k), D[k], C[k], w.intr, w.new_poses[k])
        O.integrate(int(k), w.kf_depth[k], w.kf_rgba[k], it, w.new_poses[k])
    V.check()
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny"), colour=colour,
                    c_tol=0.5 if colour == "f32" else 0.0, label=f"tiny plain update {colour}")


def test_integrate_then_deintegrate_is_exact_inverse(tinyg):
    """De-integration reverses integration (Section 4.3): with the same inputs every
    voxel returns to W = 0, D = 0, C = 0 (weights are exact integers in float32)."""
    w, D, C = tinyg
    V = gpu_volume(w, colour="rgba8")
    V.integrate(3, D[3], C[3], w.intr, w.kf_poses[3])
    e = V.extract()
    assert (e["W"] > 0).sum() > 10000
    V.deintegrate(3, D[3], C[3], w.intr, w.kf_poses[3])
    e = V.extract()
    assert torch.all(e["W"] == 0) and torch.all(e["D"] == 0) and torch.all(e["C"][..., :3] == 0)


def test_deintegrate_restores_prior_volume(tinyg):
    """Integrating keyframe 4 on top of 9 others and de-integrating it again leaves the
    other keyframes' volume (weights bit-exact, D to float rounding)."""
    w, D, C = tinyg
    A = gpu_volume(w)
    B = gpu_volume(w)
    for k in range(10):
        if k != 4:
            A.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
            B.integrate(k, D[k], C[k], w.intr, w.kf_poses[k])
    B.integrate(4, D[4], C[4], w.intr, w.kf_poses[4])
    B.deintegrate(4, D[4], C[4], w.intr, w.kf_poses[4])
    ea, eb = A.extract(), B.extract()
    ka, kb = _keys(ea["coords"].cpu().numpy()), _keys(eb["coords"].cpu().numpy())
    ia = {k: i for i, k in enumerate(ka.tolist())}
    ib = {k: i for i, k in enumerate(kb.tolist())}
    assert set(ia) <= set(ib)
    common = list(ia)
    Ia = np.array([ia[k] for k in common])
    Ib = np.array([ib[k] for k in common])
    assert torch.equal(ea["W"][Ia], eb["W"][Ib])
    assert (ea["D"][Ia] - eb["D"][Ib]).abs().max().item() < 1e-6
    extra = np.array([ib[k] for k in ib if k not in ia])
    assert torch.all(eb["W"][extra] == 0)


def test_ragged_image_and_empty_keyframe(tiny):
    """Image sizes that are not multiples of the 32x8 tile, and an all-invalid keyframe."""
    w = tiny
    d = w.kf_depth[2][:237, :301].contiguous()
    c = w.kf_rgba[2][:237, :301].contiguous()
    intr = (w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy, 301, 237)
    V = gpu_volume(w)
    V.integrate(0, d.cuda(), c.cuda(), intr, w.kf_poses[2])
    O = oracle_volume(w)
    O.integrate(0, d, c, intr, w.kf_poses[2])
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny_ragged"), label="ragged")
    E = gpu_volume(w)
    E.integrate(0, torch.zeros_like(d).cuda(), c.cuda(), intr, w.kf_poses[2])
    E.check()
    assert E.info()["allocated_blocks"] == 0
    assert E.keyframe_blocks(0).numel() == 0
    E.deintegrate(0, torch.zeros_like(d).cuda(), c.cuda(), intr, w.kf_poses[2])
    E.check()


@pytest.mark.parametrize("colour", ["f32", "rgba8"])
def test_integrate_many_matches_oracle(tinyg, colour):
    """sc_integrate_keyframes: all 10 keyframes in one graph launch."""
    w, D, C = tinyg
    it = w.intr.as_tuple()
    V = gpu_volume(w, colour=colour)
    O = oracle_volume(w, rgba8=(colour == "rgba8"))
    V.integrate_many(list(range(10)), D, C, w.kf_poses, w.intr)
    for k in range(10):
        O.integrate(k, w.kf_depth[k], w.kf_rgba[k], it, w.kf_poses[k])
    V.check()
    # RGBA8: one rounding per voxel instead of one per keyframe
    compare_volumes(V.extract(), O.export(), mu=w.trunc, max_flag_frac=flag_bound("tiny"), colour=colour,
                    c_tol=0.5 if colour == "f32" else 2.0, label=f"tiny integrate_many {colour}")
    # and the keyframes are integrated: their lists de-integrate them again
    for k in range(10):
        V.deintegrate(k, D[k], C[k], w.intr, w.kf_poses[k])
    e = V.extract()
    assert torch.all(e["W"] == 0)
