"""Shared helpers for the GPU parity tests: volume construction and the comparison of a
GPU volume with an oracle volume on the items whose decisions are not marginal."""
import numpy as np
import torch

import oracle
from paper_1709_03763_b300 import Volume


def gpu_volume(w, colour="f32", max_blocks=1 << 18, max_keyframes=64, **kw):
    return Volume(w.voxel_size, w.trunc, w.n_buckets, colour=colour, max_blocks=max_blocks,
                  max_keyframes=max_keyframes, **kw)


def oracle_volume(w, rgba8=False):
    return oracle.Volume(w.voxel_size, w.trunc, rgba8=rgba8)


def cuda(t):
    return t.contiguous().cuda()


def _keys(c):
    c = np.asarray(c, np.int64)
    return ((c[:, 0] + (1 << 20)) | ((c[:, 1] + (1 << 20)) << 21) | ((c[:, 2] + (1 << 20)) << 42))


# Share of observed voxels the oracle flags (a value-changing decision within its margin
# among the samples currently integrated, or a block whose allocation is marginal), as
# the oracle measures it on each parity workload; the tests bound it at 1.5x that.  With
# pixel coordinates spread uniformly a sample is rounding-marginal with probability
# 4 tau_px = 0.2 %, so a voxel seen by n keyframes is flagged with probability ~0.2 n %
# (Kinect-scale keyframes: ~4.5 observations per voxel -> 0.9 %).  The tiny room's
# cameras at yaw 0 and 180 deg sit on voxel lattice planes, which puts whole voxel
# planes exactly on a rounding tie (u = cx): 2-3 % of those two keyframes' voxels.
FLAG_SHARE = {
    "tiny": 0.0051,          # 10 keyframes, and after de-/re-integrating 3 of them
    "tiny_ragged": 0.0022,   # one keyframe cropped to 301 x 237
    "tiny_stream": 0.0078,   # keyframes 0-3 (keyframe 2 de-integrated) / 0-5 + a batch of 3
    "kinect6": 0.0093,       # 6 Kinect-scale keyframes, integrated and after one update
}


def flag_bound(workload: str) -> float:
    return 1.5 * FLAG_SHARE[workload]


def compare_volumes(gv: dict, ov: "oracle.Export", *, mu: float, max_flag_frac: float, colour="f32", d_tol=1e-5,
                    c_tol=0.5, rgba8_within1=0.999, label=""):
    """gv: Volume.extract() of the GPU volume; ov: oracle export; mu: truncation.  Checks
      * every robustly allocated oracle block is allocated on the GPU, and every GPU block
        is an oracle block or a marginal ("ghost") one;
      * on unflagged voxels of unflagged common blocks: W identical, |D| within d_tol,
        colour within c_tol (RGB_F32, 0..255 units) or within c_tol levels with at least
        rgba8_within1 of them within one level (RGBA8);
      * on flagged voxels (n value-changing marginal decisions among the integrated
        samples): the effect of n decisions at most -- |dW| <= n, |d(W D)| <= 2 mu n
        (d lies in [-mu, mu]) and, in RGB_F32, |d(W C)| <= 255 n, each plus the
        unflagged tolerance times W;
      * flagged voxels are at most max_flag_frac of the observed ones.
    Returns a dict of counts (the flagged share is also printed)."""
    gk = _keys(gv["coords"].cpu().numpy())
    ok = _keys(ov.coords)
    gh = set(_keys(ov.ghosts).tolist()) if len(ov.ghosts) else set()
    gidx = {k: i for i, k in enumerate(gk.tolist())}
    oidx = {k: i for i, k in enumerate(ok.tolist())}
    robust = {k for k, i in oidx.items() if ov.bflag[i] == 0}
    missing = robust - set(gidx)
    assert not missing, f"{len(missing)} robust oracle blocks not allocated on the GPU"
    extra = set(gidx) - set(oidx) - gh
    assert not extra, f"{len(extra)} GPU blocks the oracle does not allocate"
    common = [k for k in robust if k in gidx]
    G = np.array([gidx[k] for k in common])
    O = np.array([oidx[k] for k in common])
    Wg = gv["W"].cpu().numpy()[G].astype(np.float64)
    Dg = gv["D"].cpu().numpy()[G].astype(np.float64)
    Wo, Do, Co = ov.W[O], ov.D[O], ov.C[O]
    nmarg = ov.vflag[O].astype(np.float64)
    vf = nmarg != 0
    good = ~vf
    assert np.array_equal(Wg[good], Wo[good]), f"W differs on {(Wg[good] != Wo[good]).sum()} voxels"
    obs = good & (Wo > 0)
    dd = np.abs(Dg - Do)[obs]
    assert dd.max(initial=0) <= d_tol, f"max |dD| = {dd.max()}"
    assert np.all(Dg[good & (Wo == 0)] == 0)
    if colour == "f32":
        Cg = gv["C"].cpu().numpy()[G].astype(np.float64)
    else:
        Cg = gv["C"].cpu().numpy()[G][..., :3].astype(np.float64)
    dc = np.abs(Cg - Co)[obs]
    assert dc.max(initial=0) <= c_tol, f"max |dC| = {dc.max()}"
    within1 = 1.0
    if colour != "f32" and obs.any():
        within1 = float((dc.max(axis=-1) <= 1.0).mean())
        assert within1 >= rgba8_within1, f"{within1:.5f} of voxels within one colour level"
    # flagged voxels: bounded by the effect of their marginal decisions
    Wmax = np.maximum(Wg, Wo)
    n = nmarg[vf]
    assert np.all(np.abs(Wg - Wo)[vf] <= n), "W differs by more than the marginal decisions allow"
    assert np.all(np.abs(Wg * Dg - Wo * Do)[vf] <= 2 * mu * n + d_tol * Wmax[vf] + 1e-6)
    if colour == "f32":
        assert np.all(np.abs(Wg[..., None] * Cg - Wo[..., None] * Co)[vf] <=
                      (255.0 * n + c_tol * Wmax[vf] + 1e-3)[:, None])
    # flagged share: observed voxels with a marginal decision, plus every observed voxel
    # of a block whose allocation was marginal
    allW = ov.W > 0
    n_obs = int(allW.sum())
    n_flag = int((allW & ((ov.vflag != 0) | (ov.bflag[:, None] != 0))).sum())
    share = n_flag / max(n_obs, 1)
    print(f"[parity {label}] observed {n_obs}, flagged {n_flag} ({100 * share:.3f} %, bound "
          f"{100 * max_flag_frac:.3f} %), max |dD| {dd.max(initial=0):.2e}, RGBA8 within 1 level {within1:.5f}")
    assert share <= max_flag_frac, (n_flag, n_obs, max_flag_frac)
    return {"blocks": len(gk), "common": len(common), "observed": n_obs, "flagged": n_flag,
            "flag_share": share, "flagged_blocks": int((ov.bflag != 0).sum()),
            "max_dD": float(dd.max(initial=0)), "max_dC": float(dc.max(initial=0)), "within1": within1}
