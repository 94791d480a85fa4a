"""FP64 CPU oracle for keyframe surface correction (arXiv 1709.03763).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library and takes no value the CUDA path produced.

`build()` compiles surfcorr_oracle.cpp into liboracle.so (g++ -O2, FP64, IEEE
semantics, OpenMP over the blocks of one keyframe operation).  The thin ctypes
wrappers below only marshal arrays; every computation is in the C++ file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "surfcorr_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", LIB + ".tmp", SRC]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_d = ctypes.c_double
_i = ctypes.c_int
_l = ctypes.c_long
_p = ctypes.c_void_p


def _declare(L):
    L.or_fuse.argtypes = [_p, _p, _i, _p, _d, _d, _d, _d, _i, _i, _d, _p, _p, _p]
    L.or_fuse.restype = _i
    L.or_set_margins.argtypes = [_d, _d, _d]
    L.or_set_threads.argtypes = [_i]
    L.or_get_threads.restype = _i
    L.or_vol_create.argtypes = [_d, _d, _i]
    L.or_vol_create.restype = _p
    L.or_vol_destroy.argtypes = [_p]
    L.or_vol_clone.argtypes = [_p]
    L.or_vol_clone.restype = _p
    L.or_integrate.argtypes = [_p, _i, _p, _p, _d, _d, _d, _d, _i, _i, _p]
    L.or_integrate.restype = _i
    L.or_deintegrate.argtypes = [_p, _i, _p, _p, _d, _d, _d, _d, _i, _i, _p]
    L.or_deintegrate.restype = _i
    L.or_reintegrate_batch.argtypes = [_p, _i, _p, _p, _p, _p, _p, _d, _d, _d, _d, _i, _i]
    L.or_reintegrate_batch.restype = _i
    L.or_vol_num_blocks.argtypes = [_p]
    L.or_vol_num_blocks.restype = _l
    L.or_vol_export.argtypes = [_p, _p, _p, _p, _p, _p, _p]
    L.or_vol_ghosts.argtypes = [_p, _p]
    L.or_vol_ghosts.restype = _l
    L.or_vol_touched.argtypes = [_p, _i, _p, _p]
    L.or_vol_touched.restype = _l
    L.or_allocation_set.argtypes = [_d, _d, _p, _d, _d, _d, _d, _i, _i, _p, _p, _p]
    L.or_allocation_set.restype = _l
    L.or_pose_distance.argtypes = [_p, _p]
    L.or_pose_distance.restype = _d
    L.or_select_topm.argtypes = [_p, _i, _i, _p]
    L.or_select_consecutive.argtypes = [_p, _i, _i, _p]
    L.or_select_consecutive.restype = _i
    L.or_loss.argtypes = [_p, _p, _l, _d, _p, _p]
    L.or_loss.restype = _d
    L.or_grad.argtypes = [_p, _i, _p, _p, _p, _p, _d, _d, _d, _d, _i, _i, _p, _l, _d, _p, _p, _p, _p]
    L.or_grad.restype = _i
    L.or_loss_perturbed.argtypes = [_p, _i, _p, _p, _d, _d, _d, _d, _i, _i, _p, _l, _d, _p, _l, _d]
    L.or_loss_perturbed.restype = _d
    L.or_vol_stats.argtypes = [_p, _p]
    L.or_vol_export_kink.argtypes = [_p, _p]
    L.or_adjoint.argtypes = [_p, _i, _p, _p, _p, _d, _d, _d, _d, _i, _i, _l, _p, _p, _p, _p, _p, _p]
    L.or_adjoint.restype = _i
    L.or_adjoint_functional.argtypes = [_p, _i, _p, _p, _d, _d, _d, _d, _i, _i, _p, _l, _d, _l, _p, _p]
    L.or_adjoint_functional.restype = _d
    L.or_colour_unsharp.argtypes = [_p, _i, _i, _p]
    L.or_colour_blurriness.argtypes = [_p, _i, _i]
    L.or_colour_blurriness.restype = _d
    L.or_weighted_median.argtypes = [_p, _p, _i]
    L.or_weighted_median.restype = _d
    L.or_fuse_colour.argtypes = [_p, _p, _p, _i, _p, _p, _d, _d, _d, _d, _i, _i, _d, _d,
                                 _p, _p, _p, _p, _p, _p, _p]
    L.or_fuse_colour.restype = _i
    L.or_marching_cubes.argtypes = [_p, _p, _p, _l, _d, _p, _p, _l]
    L.or_marching_cubes.restype = _l
    L.or_mc_case.argtypes = [_i, _p]
    L.or_mc_case.restype = _i
    L.or_overlap.argtypes = [_p, _p, _p, _d, _d, _d, _d, _i, _i, _p]
    L.or_segment.argtypes = [_i, _d, _d, _p, _p, _i, _d, _d, _d, _d, _i, _i, _p, _p]
    L.or_segment.restype = _i
    L.or_sphere_outside.argtypes = [_p, _l, _d, _p, _d, _p, _p]
    L.or_sphere_outside.restype = _l


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.float32)


def _u8(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a), dtype=np.uint8)


def f32(x) -> float:
    """The float32 value of a parameter (the GPU library's parameters are float32;
    the oracle computes in double from exactly those values)."""
    return float(np.float32(x))


def _intr(intr):
    fx, fy, cx, cy = (f32(v) for v in tuple(intr)[:4])
    return fx, fy, cx, cy


def _np(t):
    """torch tensor or array -> numpy (host)."""
    if hasattr(t, "detach"):
        return t.detach().cpu().numpy()
    return np.asarray(t)


def set_margins(tau_px=5e-4, tau_m=2e-6, tau_rel=1e-6):
    lib().or_set_margins(tau_px, tau_m, tau_rel)


def set_threads(n: int):
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return lib().or_get_threads()


def fuse(depths, poses, kf_pose, intr, disc_rel=0.1):
    """Eq. 1 keyframe depth fusion.  depths [n,H,W] f32, poses [n,3,4], kf_pose [3,4].
    Returns (Z* [H,W] f64, W* [H,W] f64, flag [H,W] u8)."""
    d = _f32(_np(depths))
    n, H, W = d.shape
    p = _f32(_np(poses)).reshape(n, 12)
    k = _f32(_np(kf_pose)).reshape(12)
    Zs = np.zeros((H, W), np.float64)
    Ws = np.zeros((H, W), np.float64)
    fl = np.zeros((H, W), np.uint8)
    fx, fy, cx, cy = _intr(intr)
    lib().or_fuse(_ptr(d), _ptr(p), n, _ptr(k), fx, fy, cx, cy, W, H, f32(disc_rel), _ptr(Zs), _ptr(Ws), _ptr(fl))
    return Zs, Ws, fl


def unsharp(rgba):
    """Unsharp masking of one [H,W,4] uint8 image -> [H,W,3] f64 in [0, 255]."""
    c = _u8(_np(rgba))
    H, W = c.shape[:2]
    S = np.zeros((H, W, 3), np.float64)
    lib().or_colour_unsharp(_ptr(c), W, H, _ptr(S))
    return S


def blurriness(rgba) -> float:
    """Blurriness in [0, 1] of one [H,W,4] uint8 image (0 = sharp); w_b = 1 - blurriness."""
    c = _u8(_np(rgba))
    H, W = c.shape[:2]
    return lib().or_colour_blurriness(_ptr(c), W, H)


def weighted_median(values, weights) -> float:
    v = np.ascontiguousarray(values, np.float64)
    w = np.ascontiguousarray(weights, np.float64)
    return lib().or_weighted_median(_ptr(v), _ptr(w), len(v))


@dataclass
class ColourFusion:
    median: np.ndarray   # [H,W,3] f64 weighted median per channel
    err: np.ndarray      # [H,W,3] f64 bound on its move under tau_px sample moves
    rgba: np.ndarray     # [H,W,4] u8 keyframe colour C*
    nobs: np.ndarray     # [H,W] i32 observations per pixel
    wsum: np.ndarray     # [H,W] f64 total colour weight
    flag: np.ndarray     # [H,W] u8 marginal decision
    wb: np.ndarray       # [n] f64 per-frame weight w_b


def fuse_colour(rgba, depths, poses, kf_depth, kf_pose, intr, disc_rel=0.1, occl_rel=0.05) -> ColourFusion:
    """Colour keyframe fusion of frames (rgba [n,H,W,4] u8, depths [n,H,W], poses [n,3,4])
    into the keyframe with depth kf_depth [H,W] at kf_pose."""
    c = _u8(_np(rgba))
    n, H, W = c.shape[:3]
    d = _f32(_np(depths)).reshape(n, H, W)
    p = _f32(_np(poses)).reshape(n, 12)
    kd = _f32(_np(kf_depth)).reshape(H, W)
    kp = _f32(_np(kf_pose)).reshape(12)
    out = ColourFusion(np.zeros((H, W, 3)), np.zeros((H, W, 3)), np.zeros((H, W, 4), np.uint8),
                       np.zeros((H, W), np.int32), np.zeros((H, W)), np.zeros((H, W), np.uint8), np.zeros(n))
    fx, fy, cx, cy = _intr(intr)
    lib().or_fuse_colour(_ptr(c), _ptr(d), _ptr(p), n, _ptr(kd), _ptr(kp), fx, fy, cx, cy, W, H,
                         f32(disc_rel), f32(occl_rel), _ptr(out.median), _ptr(out.err), _ptr(out.rgba),
                         _ptr(out.nobs), _ptr(out.wsum), _ptr(out.flag), _ptr(out.wb))
    return out


def mc_case(mask: int) -> np.ndarray:
    """Triangles (edge triples [t,3]) of one cube whose inside corners are the bits of mask."""
    e = np.zeros((12, 3), np.int32)
    t = lib().or_mc_case(int(mask), _ptr(e))
    return e[:t].copy()


def marching_cubes(coords, D, W, voxel_size):
    """Marching Cubes over blocks (coords [n,3] int32, D, W [n,512] f32).  Returns
    (triangles [t,3,3] f64 metres, cube [t,4] int32 = first corner voxel + triangle number)."""
    c = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
    d = _f32(D).reshape(-1, 512)
    w = _f32(W).reshape(-1, 512)
    n = len(c)
    vs = f32(voxel_size)
    cnt = lib().or_marching_cubes(_ptr(c), _ptr(d), _ptr(w), n, vs, None, None, 0)
    tri = np.zeros((max(cnt, 1), 3, 3))
    cube = np.zeros((max(cnt, 1), 4), np.int32)
    lib().or_marching_cubes(_ptr(c), _ptr(d), _ptr(w), n, vs, _ptr(tri), _ptr(cube), cnt)
    return tri[:cnt], cube[:cnt]


KF_CONST, KF_DIST, KF_OVRLP = 0, 1, 2


def overlap(depth, frame_pose, kf_pose, intr):
    """Overlap counts of a frame against a keyframe: (valid, inside, marginal)."""
    d = _f32(_np(depth))
    H, W = d.shape
    c = np.zeros(3, np.int64)
    fx, fy, cx, cy = _intr(intr)
    lib().or_overlap(_ptr(d), _ptr(_f32(frame_pose).reshape(12)), _ptr(_f32(kf_pose).reshape(12)), fx, fy, cx, cy,
                     W, H, _ptr(c))
    return int(c[0]), int(c[1]), int(c[2])


def segment(strategy, params, poses, intr=None, depths=None):
    """Keyframe groups of frames in order: (frame_kf [n] int32, flag [n] u8, number of keyframes).
    KF_CONST: params = (kappa,); KF_DIST: (thr_t, thr_r); KF_OVRLP: (thr,) with depths [n,H,W]."""
    p = _f32(_np(poses)).reshape(-1, 12)
    n = len(p)
    fk = np.zeros(n, np.int32)
    fl = np.zeros(n, np.uint8)
    p0 = float(params[0])
    p1 = float(params[1]) if len(params) > 1 else 0.0
    if strategy == KF_OVRLP:
        d = _f32(_np(depths))
        H, W = d.shape[1:]
        fx, fy, cx, cy = _intr(intr)
        p0 = f32(p0)
    else:
        d, H, W, fx, fy, cx, cy = None, 0, 0, 0.0, 0.0, 0.0, 0.0
        if strategy == KF_DIST:
            p0, p1 = f32(p0), f32(p1)
    g = lib().or_segment(int(strategy), p0, p1, _ptr(d), _ptr(p), n, fx, fy, cx, cy, W, H, _ptr(fk), _ptr(fl))
    return fk, fl, g


def sphere_outside(coords, voxel_size, centre, radius):
    """Blocks outside the streaming sphere: (outside [n] bool, marginal [n] bool)."""
    c = np.ascontiguousarray(coords, np.int32).reshape(-1, 3)
    o = np.zeros(len(c), np.uint8)
    m = np.zeros(len(c), np.uint8)
    ce = np.ascontiguousarray(np.asarray(centre, np.float32).astype(np.float64))
    lib().or_sphere_outside(_ptr(c), len(c), f32(voxel_size), _ptr(ce), f32(radius), _ptr(o), _ptr(m))
    return o.astype(bool), m.astype(bool)


def allocation_set(depth, pose, intr, voxel_size, trunc):
    """A(k, T) -> (coords [n,3] int32, marginal [n] u8: 0 robust, 1 marginal member,
    2 marginal non-member)."""
    d = _f32(_np(depth))
    H, W = d.shape
    p = _f32(_np(pose)).reshape(12)
    fx, fy, cx, cy = _intr(intr)
    voxel_size, trunc = f32(voxel_size), f32(trunc)
    n = lib().or_allocation_set(voxel_size, trunc, _ptr(d), fx, fy, cx, cy, W, H, _ptr(p), None, None)
    c = np.zeros((n, 3), np.int32)
    m = np.zeros(n, np.uint8)
    lib().or_allocation_set(voxel_size, trunc, _ptr(d), fx, fy, cx, cy, W, H, _ptr(p), _ptr(c), _ptr(m))
    return c, m


@dataclass
class Export:
    coords: np.ndarray   # [n,3] int32 block coordinates, ascending key order
    D: np.ndarray        # [n,512] f64
    W: np.ndarray        # [n,512] f64
    C: np.ndarray        # [n,512,3] f64
    bflag: np.ndarray    # [n] u8
    vflag: np.ndarray    # [n,512] u8
    ghosts: np.ndarray   # [g,3] int32 blocks reached only marginally, not allocated here


class Volume:
    """Voxel-hashed TSDF in FP64.  rgba8=True stores colour as 8-bit integers."""

    def __init__(self, voxel_size, trunc, rgba8=False, _handle=None):
        voxel_size, trunc = f32(voxel_size), f32(trunc)
        self.voxel_size = voxel_size
        self.trunc = trunc
        self.rgba8 = rgba8
        self.h = _handle if _handle is not None else lib().or_vol_create(voxel_size, trunc, int(rgba8))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_vol_destroy(self.h)
            self.h = None

    def clone(self):
        return Volume(self.voxel_size, self.trunc, self.rgba8, _handle=lib().or_vol_clone(self.h))

    def integrate(self, kf_id, depth, rgba, intr, pose):
        d = _f32(_np(depth))
        H, W = d.shape
        c = _u8(_np(rgba)) if rgba is not None else None
        p = _f32(_np(pose)).reshape(12)
        fx, fy, cx, cy = _intr(intr)
        rc = lib().or_integrate(self.h, kf_id, _ptr(d), _ptr(c), fx, fy, cx, cy, W, H, _ptr(p))
        if rc:
            raise ValueError(f"keyframe {kf_id} already integrated")

    def deintegrate(self, kf_id, depth, rgba, intr, pose):
        d = _f32(_np(depth))
        H, W = d.shape
        c = _u8(_np(rgba)) if rgba is not None else None
        p = _f32(_np(pose)).reshape(12)
        fx, fy, cx, cy = _intr(intr)
        rc = lib().or_deintegrate(self.h, kf_id, _ptr(d), _ptr(c), fx, fy, cx, cy, W, H, _ptr(p))
        if rc:
            raise ValueError(f"keyframe {kf_id} not integrated")

    def reintegrate_batch(self, kf_ids, depths, rgbas, old_poses, new_poses, intr):
        ids = np.ascontiguousarray(kf_ids, np.int32)
        d = _f32(_np(depths))
        n, H, W = d.shape
        c = _u8(_np(rgbas)) if rgbas is not None else None
        op = _f32(_np(old_poses)).reshape(n, 12)
        np_ = _f32(_np(new_poses)).reshape(n, 12)
        fx, fy, cx, cy = _intr(intr)
        rc = lib().or_reintegrate_batch(self.h, n, _ptr(ids), _ptr(d), _ptr(c), _ptr(op), _ptr(np_),
                                        fx, fy, cx, cy, W, H)
        if rc:
            raise ValueError("batch item not integrated / already integrated")

    def num_blocks(self):
        return lib().or_vol_num_blocks(self.h)

    def export(self) -> Export:
        n = self.num_blocks()
        coords = np.zeros((n, 3), np.int32)
        D = np.zeros((n, 512))
        W = np.zeros((n, 512))
        C = np.zeros((n, 512, 3))
        bf = np.zeros(n, np.uint8)
        vf = np.zeros((n, 512), np.uint8)
        lib().or_vol_export(self.h, _ptr(coords), _ptr(D), _ptr(W), _ptr(C), _ptr(bf), _ptr(vf))
        g = lib().or_vol_ghosts(self.h, None)
        gh = np.zeros((g, 3), np.int32)
        lib().or_vol_ghosts(self.h, _ptr(gh))
        return Export(coords, D, W, C, bf, vf, gh)

    def touched(self, kf_id):
        n = lib().or_vol_touched(self.h, kf_id, None, None)
        if n < 0:
            return None, None
        c = np.zeros((n, 3), np.int32)
        m = np.zeros(n, np.uint8)
        lib().or_vol_touched(self.h, kf_id, _ptr(c), _ptr(m))
        return c, m

    def loss(self, points, lam=0.1):
        pts = np.ascontiguousarray(points, np.float64)
        nv = ctypes.c_long(0)
        pf = np.zeros(len(pts), np.uint8)
        L = lib().or_loss(self.h, _ptr(pts), len(pts), lam, ctypes.byref(nv), _ptr(pf))
        return L, nv.value, pf

    def grad(self, kf_ids, depths, poses, intr, points, lam=0.1, with_depth=True, with_budget=False):
        """Analytic gradient (grad_xi [K,6], grad_depth [K,H,W]); with_budget also returns the
        error budgets (err_xi [K,6], err_depth [K,H,W]) of marginal contributions."""
        ids = np.ascontiguousarray(kf_ids, np.int32)
        d = _f32(_np(depths))
        K, H, W = d.shape
        p = _f32(_np(poses)).reshape(K, 12)
        pts = np.ascontiguousarray(points, np.float64)
        gx = np.zeros((K, 6))
        gd = np.zeros((K, H, W)) if with_depth else None
        ex = np.zeros((K, 6)) if with_budget else None
        ed = np.zeros((K, H, W)) if (with_budget and with_depth) else None
        fx, fy, cx, cy = _intr(intr)
        rc = lib().or_grad(self.h, K, _ptr(ids), _ptr(d), None, _ptr(p), fx, fy, cx, cy, W, H,
                           _ptr(pts), len(pts), lam, _ptr(gx), _ptr(gd), _ptr(ex), _ptr(ed))
        if rc:
            raise ValueError("keyframe not integrated")
        if with_budget:
            return gx, gd, ex, ed
        return gx, gd

    def loss_perturbed(self, kf_id, depth, pose, intr, xi, points, lam=0.1, pix=-1, dz=0.0):
        d = _f32(_np(depth))
        H, W = d.shape
        p = _f32(_np(pose)).reshape(12)
        x = np.ascontiguousarray(xi, np.float64).reshape(6)
        pts = np.ascontiguousarray(points, np.float64)
        fx, fy, cx, cy = _intr(intr)
        return lib().or_loss_perturbed(self.h, kf_id, _ptr(d), _ptr(p), fx, fy, cx, cy, W, H, _ptr(x),
                                       int(pix), float(dz), _ptr(pts), len(pts), lam)


    def kink_flags(self) -> np.ndarray:
        """[n,512] u8 clamp-kink marginal decisions per voxel, in export() block order."""
        k = np.zeros((self.num_blocks(), 512), np.uint8)
        lib().or_vol_export_kink(self.h, _ptr(k))
        return k

    def stats(self):
        """(voxel samples in front of the camera, samples with a value-changing marginal
        decision) over every integration and de-integration of this volume."""
        out = np.zeros(2, np.int64)
        lib().or_vol_stats(self.h, _ptr(out))
        return int(out[0]), int(out[1])

    def adjoint(self, kf_ids, depths, poses, intr, g_coords, g_vals, with_depth=True):
        """Vector-Jacobian product for the cotangent G = dL/dD given per block (g_coords
        [n,3] int32, g_vals [n,512]): (grad_xi [K,6], grad_depth [K,H,W], err_xi, err_depth),
        the errors bounding what a float32 evaluation of the marginal decisions may change."""
        ids = np.ascontiguousarray(kf_ids, np.int32)
        d = _f32(_np(depths))
        K, H, W = d.shape
        p = _f32(_np(poses)).reshape(K, 12)
        gc = np.ascontiguousarray(g_coords, np.int32)
        gv = np.ascontiguousarray(g_vals, np.float64)
        gx, ex = np.zeros((K, 6)), np.zeros((K, 6))
        gd = np.zeros((K, H, W)) if with_depth else None
        ed = np.zeros((K, H, W)) if with_depth else None
        fx, fy, cx, cy = _intr(intr)
        rc = lib().or_adjoint(self.h, K, _ptr(ids), _ptr(d), _ptr(p), fx, fy, cx, cy, W, H, len(gc), _ptr(gc),
                              _ptr(gv), _ptr(gx), _ptr(gd), _ptr(ex), _ptr(ed))
        if rc:
            raise ValueError("keyframe not integrated")
        return gx, gd, ex, ed

    def adjoint_functional(self, kf_id, depth, pose, intr, xi, g_coords, g_vals, pix=-1, dz=0.0):
        """sum_v G(v) D(v) with kf_id's contribution at exp(xi^) T and depth + dz at pix, minus
        its unperturbed value, decisions frozen (for central differences of adjoint())."""
        d = _f32(_np(depth))
        H, W = d.shape
        p = _f32(_np(pose)).reshape(12)
        x = np.ascontiguousarray(xi, np.float64).reshape(6)
        gc = np.ascontiguousarray(g_coords, np.int32)
        gv = np.ascontiguousarray(g_vals, np.float64)
        fx, fy, cx, cy = _intr(intr)
        return lib().or_adjoint_functional(self.h, kf_id, _ptr(d), _ptr(p), fx, fy, cx, cy, W, H, _ptr(x), int(pix),
                                           float(dz), len(gc), _ptr(gc), _ptr(gv))


def pose_distance(T0, T1) -> float:
    a = _f32(T0).reshape(12)
    b = _f32(T1).reshape(12)
    return lib().or_pose_distance(_ptr(a), _ptr(b))


def select_topm(dist, m):
    d = np.ascontiguousarray(dist, np.float64)
    out = np.zeros(m, np.int32)
    lib().or_select_topm(_ptr(d), len(d), m, _ptr(out))
    return out


def select_consecutive(dist, m):
    d = np.ascontiguousarray(dist, np.float64)
    sums = np.zeros(max(len(d) - m + 1, 0))
    j = lib().or_select_consecutive(_ptr(d), len(d), m, _ptr(sums))
    return j, sums
