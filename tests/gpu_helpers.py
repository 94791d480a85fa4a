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


def compare_volumes(gv: dict, ov: "oracle.Export", colour="f32", d_tol=1e-5, c_tol=0.5, max_flag_frac=2e-2):
    """gv: Volume.extract() of the GPU volume; ov: oracle export.  Checks
      * every robustly allocated oracle block is allocated on the GPU, and every GPU block
        is an oracle block or a marginal ("ghost") one;
      * on unflagged voxels of unflagged common blocks: W identical, |D| within d_tol,
        colour within c_tol (RGB_F32, 0..255 units) or identical (RGBA8);
      * flagged voxels are fewer than max_flag_frac of the observed ones.
    Returns a dict of counts."""
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
    vf = ov.vflag[O] != 0
    good = ~vf
    assert np.array_equal(Wg[good], Wo[good]), f"W differs on {(Wg[good] != Wo[good]).sum()} voxels"
    obs = good & (Wo > 0)
    dd = np.abs(Dg - Do)[obs]
    assert dd.max(initial=0) <= d_tol, f"max |dD| = {dd.max()}"
    assert np.all(Dg[good & (Wo == 0)] == 0)
    if colour == "f32":
        Cg = gv["C"].cpu().numpy()[G].astype(np.float64)
        dc = np.abs(Cg - Co)[obs]
        assert dc.max(initial=0) <= c_tol, f"max |dC| = {dc.max()}"
    else:
        Cg = gv["C"].cpu().numpy()[G][..., :3].astype(np.float64)
        dc = np.abs(Cg - Co)[obs]
        assert dc.max(initial=0) <= c_tol, f"max |dC| = {dc.max()}"
    # flagged: observed voxels with a marginal decision, plus every observed voxel of a
    # block whose allocation was marginal
    allW = ov.W > 0
    n_obs = int(allW.sum())
    n_flag = int((allW & ((ov.vflag != 0) | (ov.bflag[:, None] != 0))).sum())
    assert n_flag <= max_flag_frac * max(n_obs, 1), (n_flag, n_obs)
    return {"blocks": len(gk), "common": len(common), "observed": n_obs, "flagged": n_flag,
            "flagged_blocks": int((ov.bflag != 0).sum()),
            "max_dD": float(dd.max(initial=0)), "max_dC": float(dc.max(initial=0))}
