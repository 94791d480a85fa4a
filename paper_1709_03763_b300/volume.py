"""Python binding of the surfcorr C ABI: argument marshalling over torch tensors.

Every computation runs in libsurfcorr.so's CUDA kernels; this module only checks
shapes / dtypes / devices, turns tensors into device pointers and poses into the
ABI's structs, and raises SurfcorrError on a non-zero status.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _lib
from ._lib import (BatchConfig, ColourParams, FusionParams, Intrinsics, Pose, Profile, ReintItem, SurfcorrError, VolumeInfo,
                   VolumeParams, check, lib)

__all__ = ["Volume", "BlockStore", "depth_from_u16", "fuse_frames_into_keyframe", "fuse_keyframes", "prepare_fuse", "fuse_colour_keyframes",
           "prepare_colour", "pose_distance", "select_topm", "select_consecutive",
           "pose_exp_left", "mc_case", "overlap_counts", "segment_keyframes", "KF_CONST", "KF_DIST",
           "KF_OVRLP", "SurfcorrError", "make_intrinsics", "make_pose"]


def make_intrinsics(intr) -> Intrinsics:
    """From a synthetic.Intrinsics, an Intrinsics struct or a (fx, fy, cx, cy, W, H) tuple."""
    if isinstance(intr, Intrinsics):
        return intr
    if hasattr(intr, "as_tuple"):
        intr = intr.as_tuple()
    fx, fy, cx, cy, W, H = intr
    return Intrinsics(float(fx), float(fy), float(cx), float(cy), int(W), int(H))


def make_pose(T) -> Pose:
    """[3,4] world_from_camera (numpy / torch / sequence) -> Pose struct."""
    if isinstance(T, Pose):
        return T
    if hasattr(T, "detach"):
        T = T.detach().cpu().numpy()
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float32).reshape(12))
    p = Pose()
    ctypes.memmove(ctypes.addressof(p), a.ctypes.data, 48)
    return p


def pose_array(poses):
    """Poses [n,3,4] (numpy / torch / sequence of [3,4] or Pose) as one contiguous buffer laid
    out as sc_pose[n]; returns (buffer, pointer).  Keep the buffer alive during the call."""
    n = len(poses)
    if n and isinstance(poses[0], Pose):
        buf = (Pose * n)(*poses)
        return buf, ctypes.cast(buf, ctypes.POINTER(Pose))
    if hasattr(poses, "detach"):
        poses = poses.detach().cpu().numpy()
    a = np.ascontiguousarray(np.asarray(poses, dtype=np.float32).reshape(n, 12)) if n else np.zeros((1, 12), np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(Pose))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


class Volume:
    """A voxel-hashed TSDF volume on the current CUDA device (owned by libsurfcorr)."""

    def __init__(self, voxel_size: float, trunc: float, n_buckets: int, *, bucket_size: int = 4,
                 max_blocks: int = 1 << 20, colour: str = "rgba8", max_keyframes: int = 1024,
                 max_blocks_per_keyframe: int = 1 << 16, max_batch: int = 256):
        self.colour = colour
        self.params = VolumeParams(float(voxel_size), float(trunc), int(n_buckets), int(bucket_size),
                                   int(max_blocks), _lib.SC_RGB_F32 if colour == "f32" else _lib.SC_RGBA8,
                                   int(max_keyframes), int(max_blocks_per_keyframe), int(max_batch))
        self.device = torch.cuda.current_device()
        h = ctypes.c_void_p()
        check(lib().sc_create_volume(ctypes.byref(self.params), ctypes.byref(h)), "sc_create_volume")
        self.h = h

    # -- lifetime
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sc_destroy_volume(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def voxel_size(self) -> float:
        return self.params.voxel_size

    @property
    def trunc(self) -> float:
        return self.params.trunc

    def reset(self, stream=None):
        check(lib().sc_reset_volume(self.h, _stream(stream)), "sc_reset_volume")

    def status(self) -> int:
        """Read and clear the sticky device status (0 = ok)."""
        st = ctypes.c_int32(0)
        check(lib().sc_get_status(self.h, ctypes.byref(st)), "sc_get_status")
        return st.value

    def check(self):
        st = self.status()
        if st:
            raise SurfcorrError(st, "device status")

    def info(self) -> dict:
        i = VolumeInfo()
        check(lib().sc_get_volume_info(self.h, ctypes.byref(i)), "sc_get_volume_info")
        return {k: getattr(i, k) for k, _ in VolumeInfo._fields_}

    def set_profiling(self, enabled: bool):
        check(lib().sc_set_profiling(self.h, int(bool(enabled))), "sc_set_profiling")

    def profile(self) -> dict:
        p = Profile()
        check(lib().sc_get_profile(self.h, ctypes.byref(p)), "sc_get_profile")
        return {k: getattr(p, k) for k, _ in Profile._fields_ if k != "pad"}

    def set_retry_limit(self, n: int):
        check(lib().sc_set_retry_limit(self.h, int(n)), "sc_set_retry_limit")

    # -- plain path
    def integrate(self, kf_id: int, depth: torch.Tensor, rgba: torch.Tensor, intr, pose, stream=None):
        check(lib().sc_integrate_keyframe(self.h, int(kf_id), _dev(depth, torch.float32, "depth"),
                                          _dev(rgba, torch.uint8, "rgba"), ctypes.byref(make_intrinsics(intr)),
                                          ctypes.byref(make_pose(pose)), _stream(stream)),
              "sc_integrate_keyframe")

    def deintegrate(self, kf_id: int, depth: torch.Tensor, rgba: torch.Tensor, intr, pose, stream=None):
        check(lib().sc_deintegrate_keyframe(self.h, int(kf_id), _dev(depth, torch.float32, "depth"),
                                            _dev(rgba, torch.uint8, "rgba"), ctypes.byref(make_intrinsics(intr)),
                                            ctypes.byref(make_pose(pose)), _stream(stream)),
              "sc_deintegrate_keyframe")

    # -- batched path
    @staticmethod
    def prepare_integrate_many(kf_ids: Sequence[int], depths, rgbas, poses):
        """Argument arrays for integrate_many, built once and reusable (the tensors must stay alive)."""
        n = len(kf_ids)
        ids = (ctypes.c_int32 * n)(*[int(k) for k in kf_ids])
        dp = (ctypes.c_void_p * n)(*[_dev(depths[i], torch.float32, "depth") for i in range(n)])
        cp = (ctypes.c_void_p * n)(*[_dev(rgbas[i], torch.uint8, "rgba") for i in range(n)])
        pz = (Pose * n)(*[make_pose(p) for p in poses])
        return (n, ids, dp, cp, pz)

    def integrate_many(self, kf_ids: Sequence[int] = None, depths=None, rgbas=None, poses=None, intr=None,
                       stream=None, prepared=None):
        """Integrate several not-yet-integrated keyframes in one graph launch."""
        n, ids, dp, cp, pz = prepared if prepared is not None else self.prepare_integrate_many(kf_ids, depths, rgbas,
                                                                                              poses)
        check(lib().sc_integrate_keyframes(self.h, ids, dp, cp, pz, n, ctypes.byref(make_intrinsics(intr)),
                                           _stream(stream)), "sc_integrate_keyframes")

    def _items(self, kf_ids, depths, rgbas, old_poses, new_poses):
        n = len(kf_ids)
        arr = (ReintItem * n)()
        for i in range(n):
            d = depths[i]
            c = rgbas[i]
            arr[i].depth = _dev(d, torch.float32, "depth")
            arr[i].rgba = _dev(c, torch.uint8, "rgba")
            arr[i].old_pose = make_pose(old_poses[i])
            arr[i].new_pose = make_pose(new_poses[i])
            arr[i].kf_id = int(kf_ids[i])
        return arr

    def prepare_batch(self, kf_ids: Sequence[int], depths, rgbas, old_poses, new_poses):
        """The item array of reintegrate_batch, built once and reusable."""
        return self._items(kf_ids, depths, rgbas, old_poses, new_poses)

    def reintegrate_batch(self, kf_ids: Sequence[int] = None, depths=None, rgbas=None, old_poses=None,
                          new_poses=None, intr=None, stream=None, prepared=None):
        """One pose-graph update: de-integrate each keyframe at its old pose and re-integrate at
        its new pose (one graph launch).  depths / rgbas: tensors [n,H,W] / [n,H,W,4] or lists."""
        arr = prepared if prepared is not None else self._items(kf_ids, depths, rgbas, old_poses, new_poses)
        check(lib().sc_reintegrate_batch(self.h, arr, len(arr), ctypes.byref(make_intrinsics(intr)),
                                         _stream(stream)), "sc_reintegrate_batch")

    def set_batch_config(self, warps_per_cta=4, ctas_per_sm=8, blocks_per_grab=1):
        c = BatchConfig(warps_per_cta, ctas_per_sm, blocks_per_grab)
        check(lib().sc_set_batch_config(self.h, ctypes.byref(c)), "sc_set_batch_config")

    def batch_config(self) -> dict:
        c = BatchConfig()
        check(lib().sc_get_batch_config(self.h, ctypes.byref(c)), "sc_get_batch_config")
        return {k: getattr(c, k) for k, _ in BatchConfig._fields_}

    def autotune_batch(self, kf_ids, depths, rgbas, old_poses, new_poses, intr, stream=None):
        arr = self._items(kf_ids, depths, rgbas, old_poses, new_poses)
        best = BatchConfig()
        ms = ctypes.c_float(0)
        check(lib().sc_autotune_batch(self.h, arr, len(kf_ids), ctypes.byref(make_intrinsics(intr)),
                                      _stream(stream), ctypes.byref(best), ctypes.byref(ms)), "sc_autotune_batch")
        return {k: getattr(best, k) for k, _ in BatchConfig._fields_}, ms.value

    # -- extraction
    def extract(self, payload: bool = True, capacity: int | None = None, stream=None) -> dict:
        """Allocated blocks: coords [n,3] int32, slots [n] int32 and, with payload, D / W [n,512]
        float32 and C [n,512,4] uint8 (rgba8) or [n,512,3] float32 (f32).  Unordered."""
        cap = int(capacity if capacity is not None else self.info()["allocated_blocks"])
        dev = torch.device("cuda", self.device)
        coords = torch.empty((max(cap, 1), 3), dtype=torch.int32, device=dev)
        slots = torch.empty((max(cap, 1),), dtype=torch.int32, device=dev)
        D = W = C = None
        if payload:
            D = torch.empty((max(cap, 1), 512), dtype=torch.float32, device=dev)
            W = torch.empty_like(D)
            C = (torch.empty((max(cap, 1), 512, 3), dtype=torch.float32, device=dev) if self.colour == "f32"
                 else torch.empty((max(cap, 1), 512, 4), dtype=torch.uint8, device=dev))
        n = ctypes.c_int32(0)
        rc = lib().sc_extract_block_list(self.h, coords.data_ptr(), slots.data_ptr(),
                                         D.data_ptr() if payload else None, W.data_ptr() if payload else None,
                                         C.data_ptr() if payload else None, cap, ctypes.byref(n), _stream(stream))
        check(rc, "sc_extract_block_list")
        m = n.value
        out = {"coords": coords[:m], "slots": slots[:m]}
        if payload:
            out.update(D=D[:m], W=W[:m], C=C[:m])
        return out

    def import_blocks(self, coords: torch.Tensor, D: torch.Tensor, W: torch.Tensor, C: torch.Tensor | None = None,
                      stream=None):
        """Insert / overwrite blocks: coords [n,3] int32, D / W [n,512] float32, C [n,512,4] uint8
        (rgba8) or [n,3,512] float32 (f32) or None (device tensors)."""
        n = int(coords.shape[0])
        if n == 0:
            return
        if D.shape != (n, 512) or W.shape != (n, 512):
            raise ValueError("D and W must be [n, 512]")
        cptr = None
        if C is not None:
            cptr = (_dev(C, torch.float32, "C") if self.colour == "f32" else _dev(C, torch.uint8, "C"))
            if C.numel() != n * 512 * (3 if self.colour == "f32" else 4):
                raise ValueError("C has the wrong size for the volume's colour format")
        check(lib().sc_import_blocks(self.h, _dev(coords, torch.int32, "coords"), _dev(D, torch.float32, "D"),
                                     _dev(W, torch.float32, "W"), cptr, n, _stream(stream)), "sc_import_blocks")

    def set_keyframe_blocks(self, kf_id: int, coords: torch.Tensor, stream=None):
        """Restore keyframe kf_id's block list from block coordinates [n,3] int32 (device)."""
        n = int(coords.shape[0])
        ptr = _dev(coords.contiguous(), torch.int32, "coords") if n else None
        check(lib().sc_set_keyframe_blocks(self.h, int(kf_id), ptr, n, _stream(stream)), "sc_set_keyframe_blocks")

    def save(self, path: str, keyframes=()):
        """Checkpoint: every block (coords, D, W, C) and the block lists (as coordinates)
        of the given integrated keyframes, to an .npz file."""
        ex = self.extract()
        out = {k: v.cpu().numpy() for k, v in ex.items()}
        slot_coord = {}
        slots = ex["slots"].cpu().numpy()
        coords = out["coords"]
        idx = np.full(int(slots.max()) + 1 if len(slots) else 1, -1, np.int64)
        idx[slots] = np.arange(len(slots))
        for k in keyframes:
            ks = self.keyframe_blocks(int(k)).cpu().numpy()
            out[f"kf_{int(k)}"] = coords[idx[ks]]
        out["colour"] = np.array(self.colour)
        np.savez(path, **out)

    def load(self, path: str, stream=None) -> list:
        """Resume from save(): import the blocks into this (empty) volume and restore the
        saved keyframes' block lists.  Returns the restored keyframe ids."""
        z = np.load(path)
        if str(z["colour"]) != self.colour:
            raise ValueError("checkpoint colour format differs from the volume's")
        dev = torch.device("cuda", self.device)
        C = torch.from_numpy(z["C"]).to(dev)
        if self.colour == "f32":
            C = C.permute(0, 2, 1).contiguous()  # extract gives [n,512,3]; import takes [n,3,512]
        else:
            C = C.contiguous()
        self.import_blocks(torch.from_numpy(z["coords"]).to(dev), torch.from_numpy(z["D"]).to(dev),
                           torch.from_numpy(z["W"]).to(dev), C, stream=stream)
        kfs = sorted(int(k[3:]) for k in z.files if k.startswith("kf_"))
        for k in kfs:
            self.set_keyframe_blocks(k, torch.from_numpy(z[f"kf_{k}"]).to(dev), stream=stream)
        return kfs

    def marching_cubes(self, capacity: int | None = None, cubes: bool = False, out: torch.Tensor | None = None,
                       stream=None):
        """Zero-level-set triangles [t,3,3] float32 (metres) and, with cubes=True, their cube
        ids [t,4] int32 (first corner voxel, triangle number in the cube).  Unordered.
        Without a capacity the call counts first, then extracts."""
        dev = torch.device("cuda", self.device)
        n = ctypes.c_int64(0)
        if capacity is None and out is None:
            rc = lib().sc_marching_cubes(self.h, None, None, 0, ctypes.byref(n), _stream(stream))
            if rc not in (_lib.SC_OK, _lib.SC_ERR_CAPACITY):
                check(rc, "sc_marching_cubes")
            capacity = n.value
        if out is None:
            out = torch.empty((max(int(capacity), 1), 3, 3), dtype=torch.float32, device=dev)
        cap = out.shape[0] if capacity is None else int(capacity)
        cb = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=dev) if cubes else None
        check(lib().sc_marching_cubes(self.h, _dev(out, torch.float32, "out"), cb.data_ptr() if cubes else None,
                                      cap, ctypes.byref(n), _stream(stream)), "sc_marching_cubes")
        t = n.value
        return (out[:t], cb[:t]) if cubes else out[:t]

    def stream_out(self, store: "BlockStore", centre, radius: float, stream=None) -> int:
        """Move the blocks whose centre is farther than radius from centre into the host
        store; returns the number moved."""
        c = (ctypes.c_float * 3)(*[float(x) for x in np.asarray(centre).reshape(3)])
        n = ctypes.c_int64(0)
        check(lib().sc_stream_out(self.h, store.h, c, float(radius), ctypes.byref(n), _stream(stream)),
              "sc_stream_out")
        return n.value

    def stream_in(self, store: "BlockStore", centre, radius: float = float("inf"), stream=None) -> int:
        """Move the stored blocks whose centre is within radius of centre back to the GPU;
        returns the number moved."""
        c = (ctypes.c_float * 3)(*[float(x) for x in np.asarray(centre).reshape(3)])
        n = ctypes.c_int64(0)
        check(lib().sc_stream_in(self.h, store.h, c, float(radius), ctypes.byref(n), _stream(stream)),
              "sc_stream_in")
        return n.value

    def stream_in_keyframes(self, store: "BlockStore", kf_ids, stream=None) -> int:
        """Move the stored blocks that the keyframes' block lists name back to the GPU."""
        ids = (ctypes.c_int32 * max(len(kf_ids), 1))(*[int(k) for k in kf_ids])
        n = ctypes.c_int64(0)
        check(lib().sc_stream_in_keyframes(self.h, store.h, ids, len(kf_ids), ctypes.byref(n), _stream(stream)),
              "sc_stream_in_keyframes")
        return n.value

    def stream_in_poses(self, store: "BlockStore", depths, poses, intr, stream=None) -> int:
        """Move back the stored blocks that allocating A(k, T) for these keyframe depth
        images (device [n,H,W] or a list) at these poses would reach."""
        n = len(poses)
        dp = (ctypes.c_void_p * max(n, 1))(*[_dev(depths[i], torch.float32, "depth") for i in range(n)])
        pz = (Pose * max(n, 1))(*[make_pose(p) for p in poses])
        moved = ctypes.c_int64(0)
        check(lib().sc_stream_in_poses(self.h, store.h, dp, pz, n, ctypes.byref(make_intrinsics(intr)),
                                       ctypes.byref(moved), _stream(stream)), "sc_stream_in_poses")
        return moved.value

    def keyframe_blocks(self, kf_id: int, stream=None) -> torch.Tensor:
        """Pool slots of kf_id's stored block list (its allocation set A(k, T))."""
        n = ctypes.c_int32(0)
        rc = lib().sc_get_keyframe_blocks(self.h, int(kf_id), None, 0, ctypes.byref(n), _stream(stream))
        if rc not in (_lib.SC_OK, _lib.SC_ERR_CAPACITY):
            check(rc, "sc_get_keyframe_blocks")
        out = torch.empty((max(n.value, 1),), dtype=torch.int32, device=torch.device("cuda", self.device))
        check(lib().sc_get_keyframe_blocks(self.h, int(kf_id), out.data_ptr(), n.value, ctypes.byref(n),
                                           _stream(stream)), "sc_get_keyframe_blocks")
        return out[:n.value]

    # -- loss and adjoint
    def grad_buffer(self) -> torch.Tensor:
        return torch.zeros((self.params.max_blocks, 512), dtype=torch.float32,
                           device=torch.device("cuda", self.device))

    def sdf_loss(self, points: torch.Tensor, lam: float = 0.1, grad_D: torch.Tensor | None = None, stream=None,
                 out: torch.Tensor | None = None):
        """Returns (out [5] float64 device: L, P, sum Dt^2, sum W D^2, sum W;  grad_D)."""
        if grad_D is None:
            grad_D = self.grad_buffer()
        if out is None:
            out = torch.empty(5, dtype=torch.float64, device=torch.device("cuda", self.device))
        pts = points
        check(lib().sc_sdf_loss(self.h, _dev(pts, torch.float32, "points"), int(pts.shape[0]), float(lam),
                                _dev(grad_D, torch.float32, "grad_D"), out.data_ptr(), _stream(stream)),
              "sc_sdf_loss")
        return out, grad_D

    @staticmethod
    def prepare_adjoint(kf_ids, depths, poses):
        """Argument arrays for sdf_adjoint, built once and reusable."""
        n = len(kf_ids)
        ids = (ctypes.c_int32 * n)(*[int(k) for k in kf_ids])
        ptrs = (ctypes.c_void_p * n)(*[_dev(depths[i], torch.float32, "depth") for i in range(n)])
        pz = (Pose * n)(*[make_pose(poses[i]) for i in range(n)])
        return (n, ids, ptrs, pz)

    def sdf_adjoint(self, kf_ids=None, depths=None, poses=None, intr=None, grad_D=None, with_depth=True,
                    stream=None, prepared=None, out=None):
        """Gradient of the loss w.r.t. each keyframe's left se(3) pose perturbation
        (grad_xi [n,6] float64) and its depth pixels (grad_depth [n,H,W] float32).
        out: optional preallocated (grad_xi, grad_depth)."""
        n, ids, ptrs, pz = prepared if prepared is not None else self.prepare_adjoint(kf_ids, depths, poses)
        K = make_intrinsics(intr)
        dev = torch.device("cuda", self.device)
        if out is not None:
            gx, gd = out
        else:
            gx = torch.empty((n, 6), dtype=torch.float64, device=dev)
            gd = torch.empty((n, K.height, K.width), dtype=torch.float32, device=dev) if with_depth else None
        check(lib().sc_sdf_adjoint(self.h, ids, ptrs, pz, n, ctypes.byref(K), _dev(grad_D, torch.float32, "grad_D"),
                                   gx.data_ptr(), gd.data_ptr() if with_depth else None, _stream(stream)),
              "sc_sdf_adjoint")
        return gx, gd


def fuse_frames_into_keyframe(depths: torch.Tensor, frame_poses, kf_pose, intr, disc_rel: float = 0.1,
                              out_depth: torch.Tensor | None = None, out_weight: torch.Tensor | None = None,
                              stream=None):
    """Eq. 1 keyframe depth fusion of frames [n,H,W] into the keyframe pose.  Returns (Z*, W*)."""
    n, H, W = depths.shape
    if out_depth is None:
        out_depth = torch.empty((H, W), dtype=torch.float32, device=depths.device)
    if out_weight is None:
        out_weight = torch.empty((H, W), dtype=torch.float32, device=depths.device)
    pz = (Pose * n)(*[make_pose(p) for p in frame_poses])
    fp = FusionParams(float(disc_rel))
    check(lib().sc_fuse_frames_into_keyframe(_dev(depths, torch.float32, "depths"), pz, n,
                                             ctypes.byref(make_pose(kf_pose)), ctypes.byref(make_intrinsics(intr)),
                                             ctypes.byref(fp), _dev(out_depth, torch.float32, "out_depth"),
                                             _dev(out_weight, torch.float32, "out_weight"), _stream(stream)),
          "sc_fuse_frames_into_keyframe")
    return out_depth, out_weight


def prepare_fuse(frame_poses, frame_kf, kf_poses):
    """Argument arrays for fuse_keyframes, built once and reusable."""
    n, n_kf = len(frame_poses), len(kf_poses)
    pz = (Pose * n)(*[make_pose(p) for p in frame_poses])
    kz = (Pose * n_kf)(*[make_pose(p) for p in kf_poses])
    fk = (ctypes.c_int32 * n)(*[int(k) for k in frame_kf])
    return (pz, fk, kz)


def fuse_keyframes(depths: torch.Tensor, frame_poses=None, frame_kf=None, kf_poses=None, intr=None,
                   disc_rel: float = 0.1, out_depth: torch.Tensor | None = None,
                   out_weight: torch.Tensor | None = None, stream=None, prepared=None):
    """Eq. 1 for many keyframes in one call: frame f is fused into keyframe frame_kf[f].
    depths [n,H,W]; returns (Z* [n_kf,H,W], W* [n_kf,H,W])."""
    pz, fk, kz = prepared if prepared is not None else prepare_fuse(frame_poses, frame_kf, kf_poses)
    n, H, W = depths.shape
    n_kf = len(kz)
    if len(pz) != n:
        raise ValueError("frame pose count does not match the depth frames")
    if out_depth is None:
        out_depth = torch.empty((n_kf, H, W), dtype=torch.float32, device=depths.device)
    if out_weight is None:
        out_weight = torch.empty((n_kf, H, W), dtype=torch.float32, device=depths.device)
    fp = FusionParams(float(disc_rel))
    check(lib().sc_fuse_keyframes(_dev(depths, torch.float32, "depths"), pz, fk, n, kz, n_kf,
                                  ctypes.byref(make_intrinsics(intr)), ctypes.byref(fp),
                                  _dev(out_depth, torch.float32, "out_depth"),
                                  _dev(out_weight, torch.float32, "out_weight"), _stream(stream)),
          "sc_fuse_keyframes")
    return out_depth, out_weight


def depth_from_u16(raw: torch.Tensor, scale: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Raw 16-bit sensor depth (any shape, int16 / uint16 storage) to metres: raw * scale."""
    if raw.dtype not in (torch.int16, torch.uint16):
        raise TypeError("raw depth must be 16-bit")
    if not raw.is_cuda or not raw.is_contiguous():
        raise ValueError("raw depth must be a contiguous CUDA tensor")
    if out is None:
        out = torch.empty(raw.shape, dtype=torch.float32, device=raw.device)
    check(lib().sc_depth_from_u16(raw.data_ptr(), raw.numel(), float(scale), _dev(out, torch.float32, "out"),
                                  _stream(stream)), "sc_depth_from_u16")
    return out


def rgba_from_rgb(rgb: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Packed RGB8 images [..., 3] (uint8, CUDA) to RGBA8 [..., 4] with alpha 255."""
    if rgb.dtype != torch.uint8 or rgb.shape[-1] != 3:
        raise TypeError("rgb must be uint8 with a last dimension of 3")
    if not rgb.is_cuda or not rgb.is_contiguous():
        raise ValueError("rgb must be a contiguous CUDA tensor")
    if out is None:
        out = torch.empty((*rgb.shape[:-1], 4), dtype=torch.uint8, device=rgb.device)
    if out.dtype != torch.uint8 or out.numel() != 4 * (rgb.numel() // 3) or not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor of 4 bytes a pixel")
    check(lib().sc_rgba_from_rgb(rgb.data_ptr(), rgb.numel() // 3, out.data_ptr(), _stream(stream)),
          "sc_rgba_from_rgb")
    return out


def prepare_colour(frame_poses, frame_kf, kf_poses, width: int, height: int, device=None):
    """Argument arrays and the device workspace for fuse_colour_keyframes, built once
    and reusable (the workspace must not be shared by calls that overlap on the GPU)."""
    n, n_kf = len(frame_poses), len(kf_poses)
    pz = (Pose * n)(*[make_pose(p) for p in frame_poses])
    kz = (Pose * n_kf)(*[make_pose(p) for p in kf_poses])
    fk = (ctypes.c_int32 * n)(*[int(k) for k in frame_kf])
    nbytes = int(lib().sc_colour_workspace_bytes(int(width), int(height)))
    if nbytes == 0:
        raise ValueError("image size out of range for colour fusion")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device if device is not None else torch.cuda.current_device())
    return (pz, fk, kz, ws)


def fuse_colour_keyframes(rgba: torch.Tensor, depths: torch.Tensor, kf_depth: torch.Tensor, frame_poses=None,
                          frame_kf=None, kf_poses=None, intr=None, disc_rel: float = 0.1, occl_rel: float = 0.05,
                          out_rgba: torch.Tensor | None = None, out_colour: torch.Tensor | bool | None = None,
                          out_weight: torch.Tensor | bool | None = None, stream=None, prepared=None):
    """Colour keyframe fusion (unsharp masking, blurriness weight, back-warp with bilinear
    sampling, weighted median) of frames rgba [n,H,W,4] u8 / depths [n,H,W] into the
    keyframes with depth kf_depth [n_kf,H,W].  Returns (C* [n_kf,H,W,4] u8, medians
    [n_kf,H,W,3] f32 or None, w_b [n] f32 or None); out_colour / out_weight = True
    allocate those outputs."""
    n, H, W = depths.shape
    if prepared is None:
        prepared = prepare_colour(frame_poses, frame_kf, kf_poses, W, H, depths.device)
    pz, fk, kz, ws = prepared
    n_kf = len(kz)
    if len(pz) != n or rgba.shape != (n, H, W, 4) or kf_depth.shape != (n_kf, H, W):
        raise ValueError("frame / keyframe shapes do not match")
    if out_rgba is None:
        out_rgba = torch.empty((n_kf, H, W, 4), dtype=torch.uint8, device=depths.device)
    if out_colour is True:
        out_colour = torch.empty((n_kf, H, W, 3), dtype=torch.float32, device=depths.device)
    if out_weight is True:
        out_weight = torch.empty(n, dtype=torch.float32, device=depths.device)
    cp = ColourParams(float(disc_rel), float(occl_rel))
    col_ptr = _dev(out_colour, torch.float32, "out_colour") if isinstance(out_colour, torch.Tensor) else None
    w_ptr = _dev(out_weight, torch.float32, "out_weight") if isinstance(out_weight, torch.Tensor) else None
    check(lib().sc_fuse_colour_keyframes(_dev(rgba, torch.uint8, "rgba"), _dev(depths, torch.float32, "depths"),
                                         pz, fk, n, _dev(kf_depth, torch.float32, "kf_depth"), kz, n_kf,
                                         ctypes.byref(make_intrinsics(intr)), ctypes.byref(cp),
                                         _dev(ws, torch.uint8, "workspace"), ws.numel(),
                                         _dev(out_rgba, torch.uint8, "out_rgba"), col_ptr, w_ptr, _stream(stream)),
          "sc_fuse_colour_keyframes")
    return (out_rgba, out_colour if isinstance(out_colour, torch.Tensor) else None,
            out_weight if isinstance(out_weight, torch.Tensor) else None)


def fusion_profile(enable: int = -1) -> dict:
    """Fusion launch timing: enable=1 resets and starts, 0 resets and stops, -1 reads."""
    ms = ctypes.c_double(0)
    n = ctypes.c_int64(0)
    f = ctypes.c_int64(0)
    check(lib().sc_fusion_profile(int(enable), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(f)),
          "sc_fusion_profile")
    return {"ms": ms.value, "launches": n.value, "frames": f.value}


def pose_distance(a, b) -> float:
    pa, pb = make_pose(a), make_pose(b)
    return lib().sc_pose_distance(ctypes.byref(pa), ctypes.byref(pb))


def select_topm(dist, m: int) -> np.ndarray:
    d = np.ascontiguousarray(dist, np.float64)
    out = np.zeros(min(m, len(d)), np.int32)
    check(lib().sc_select_topm(d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(d), int(m),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "sc_select_topm")
    return out


def select_consecutive(dist, m: int) -> int:
    d = np.ascontiguousarray(dist, np.float64)
    j = lib().sc_select_consecutive(d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(d), int(m))
    if j < 0:
        raise SurfcorrError(j, "sc_select_consecutive")
    return j


KF_CONST, KF_DIST, KF_OVRLP = _lib.SC_KF_CONST, _lib.SC_KF_DIST, _lib.SC_KF_OVRLP


def overlap_counts(depths: torch.Tensor, frame_poses, kf_pose, intr, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """KF_OVRLP counts [n,2] int64 (valid pixels, overlapping pixels) of frames against a keyframe."""
    n = depths.shape[0]
    if out is None:
        out = torch.empty((max(n, 1), 2), dtype=torch.int64, device=depths.device)
    pz = (Pose * max(n, 1))(*[make_pose(p) for p in frame_poses])
    check(lib().sc_overlap_counts(_dev(depths, torch.float32, "depths"), pz, n, ctypes.byref(make_pose(kf_pose)),
                                  ctypes.byref(make_intrinsics(intr)), _dev(out, torch.int64, "out"),
                                  _stream(stream)), "sc_overlap_counts")
    return out[:n]


def segment_keyframes(strategy: int, params, poses, intr=None, depths: torch.Tensor | None = None,
                      stream=None) -> tuple[np.ndarray, int]:
    """Keyframe groups of frames in order (KF_CONST: params=(kappa,), KF_DIST: (thr_t, thr_r),
    KF_OVRLP: (thr,) with depths [n,H,W] on the device).  Returns (frame_kf [n] int32, keyframes)."""
    n = len(poses)
    pbuf, pz = pose_array(poses)
    pr = (ctypes.c_double * 2)(*[float(x) for x in (list(params) + [0.0, 0.0])[:2]])
    fk = np.zeros(max(n, 1), np.int32)
    g = ctypes.c_int32(0)
    dptr = _dev(depths, torch.float32, "depths") if depths is not None else None
    iptr = ctypes.byref(make_intrinsics(intr)) if intr is not None else None
    # KF_CONST / KF_DIST run on the host only: no stream needed
    st = _stream(stream) if (depths is not None or stream is not None) else None
    check(lib().sc_segment_keyframes(int(strategy), pr, dptr, pz, n, iptr,
                                     fk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(g), st),
          "sc_segment_keyframes")
    return fk[:n], g.value


class BlockStore:
    """Host block store of the streaming sphere (pinned, device-mapped memory)."""

    def __init__(self, capacity: int, colour: str = "rgba8"):
        self.h = ctypes.c_void_p()
        check(lib().sc_create_block_store(int(capacity), _lib.SC_RGB_F32 if colour == "f32" else _lib.SC_RGBA8,
                                          ctypes.byref(self.h)), "sc_create_block_store")

    def __len__(self) -> int:
        return int(lib().sc_block_store_count(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sc_destroy_block_store(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_case(mask: int) -> np.ndarray:
    """The library's Marching Cubes triangulation of an inside-corner mask: edge triples [t,3]."""
    e = (ctypes.c_int32 * 15)()
    t = lib().sc_mc_case(int(mask), e)
    if t < 0:
        raise SurfcorrError(t, "sc_mc_case")
    return np.array(list(e)[:3 * t], dtype=np.int32).reshape(t, 3)


def pose_exp_left(T, xi) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(xi, np.float64).reshape(6))
    out = Pose()
    check(lib().sc_pose_exp_left(ctypes.byref(make_pose(T)), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.byref(out)), "sc_pose_exp_left")
    return np.array(out.m, dtype=np.float32).reshape(3, 4)
