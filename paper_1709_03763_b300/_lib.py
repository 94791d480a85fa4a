"""ctypes declarations for libsurfcorr.so (the C ABI in include/surfcorr.h).

Argument marshalling only.  The library is loaded from this package directory;
if it is missing the import fails loudly (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsurfcorr.so")

c_f = ctypes.c_float
c_d = ctypes.c_double
c_i32 = ctypes.c_int32
c_u32 = ctypes.c_uint32
c_i64 = ctypes.c_int64
c_u64 = ctypes.c_uint64
c_p = ctypes.c_void_p

SC_OK = 0
SC_ERR_INVALID_ARG = -1
SC_ERR_CUDA = -2
SC_ERR_HASH_FULL = -3
SC_ERR_POOL_FULL = -4
SC_ERR_RETRY_LIMIT = -5
SC_ERR_NOT_INTEGRATED = -6
SC_ERR_CAPACITY = -7
SC_ERR_ALREADY_INTEGRATED = -8
SC_ERR_LIST_FULL = -9
SC_ERR_NOT_RESIDENT = -10
SC_ERR_CONFLICT = -11
SC_RGBA8 = 0
SC_RGB_F32 = 1


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f), ("width", c_i32), ("height", c_i32)]


class Pose(ctypes.Structure):
    _fields_ = [("m", c_f * 12)]


class VolumeParams(ctypes.Structure):
    _fields_ = [("voxel_size", c_f), ("trunc", c_f), ("n_buckets", c_u32), ("bucket_size", c_u32),
                ("max_blocks", c_u32), ("colour_format", c_i32), ("max_keyframes", c_i32),
                ("max_blocks_per_keyframe", c_u32), ("max_batch", c_i32)]


class FusionParams(ctypes.Structure):
    _fields_ = [("disc_rel", c_f)]


SC_KF_CONST, SC_KF_DIST, SC_KF_OVRLP = 0, 1, 2


class ColourParams(ctypes.Structure):
    _fields_ = [("disc_rel", c_f), ("occl_rel", c_f)]


class ReintItem(ctypes.Structure):
    _fields_ = [("depth", c_p), ("rgba", c_p), ("old_pose", Pose), ("new_pose", Pose), ("kf_id", c_i32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("warps_per_cta", c_i32), ("ctas_per_sm", c_i32), ("blocks_per_grab", c_i32)]


class VolumeInfo(ctypes.Structure):
    _fields_ = [("allocated_blocks", c_u32), ("max_blocks", c_u32), ("hash_entries", c_u32),
                ("integrated_keyframes", c_i32), ("device_bytes", c_u64)]


class Profile(ctypes.Structure):
    _fields_ = [("enabled", c_i32), ("pad", c_i32), ("alloc_ms", c_d), ("alloc_launches", c_i64),
                ("update_ms", c_d), ("update_launches", c_i64), ("update_blocks", c_i64),
                ("batch_alloc_ms", c_d), ("batch_mark_ms", c_d), ("batch_net_ms", c_d),
                ("batch_launches", c_i64), ("batch_union_blocks", c_i64), ("batch_pairs", c_i64),
                ("mc_ms", c_d), ("mc_launches", c_i64)]


P = ctypes.POINTER

# name -> (restype, argtypes); every symbol declared in include/surfcorr.h
SIGNATURES = {
    "sc_create_volume": (c_i32, [P(VolumeParams), P(c_p)]),
    "sc_destroy_volume": (c_i32, [c_p]),
    "sc_reset_volume": (c_i32, [c_p, c_p]),
    "sc_get_status": (c_i32, [c_p, P(c_i32)]),
    "sc_get_volume_info": (c_i32, [c_p, P(VolumeInfo)]),
    "sc_status_string": (ctypes.c_char_p, [c_i32]),
    "sc_fuse_frames_into_keyframe": (c_i32, [c_p, P(Pose), c_i32, P(Pose), P(Intrinsics), P(FusionParams),
                                             c_p, c_p, c_p]),
    "sc_fuse_keyframes": (c_i32, [c_p, P(Pose), P(c_i32), c_i32, P(Pose), c_i32, P(Intrinsics), P(FusionParams),
                                  c_p, c_p, c_p]),
    "sc_depth_from_u16": (c_i32, [c_p, c_i64, c_f, c_p, c_p]),
    "sc_rgba_from_rgb": (c_i32, [c_p, c_i64, c_p, c_p]),
    "sc_colour_workspace_bytes": (c_u64, [c_i32, c_i32]),
    "sc_fuse_colour_keyframes": (c_i32, [c_p, c_p, P(Pose), P(c_i32), c_i32, c_p, P(Pose), c_i32, P(Intrinsics),
                                         P(ColourParams), c_p, c_u64, c_p, c_p, c_p, c_p]),
    "sc_overlap_counts": (c_i32, [c_p, P(Pose), c_i32, P(Pose), P(Intrinsics), c_p, c_p]),
    "sc_segment_keyframes": (c_i32, [c_i32, P(c_d), c_p, P(Pose), c_i32, P(Intrinsics), P(c_i32), P(c_i32), c_p]),
    "sc_integrate_keyframe": (c_i32, [c_p, c_i32, c_p, c_p, P(Intrinsics), P(Pose), c_p]),
    "sc_deintegrate_keyframe": (c_i32, [c_p, c_i32, c_p, c_p, P(Intrinsics), P(Pose), c_p]),
    "sc_reintegrate_batch": (c_i32, [c_p, P(ReintItem), c_i32, P(Intrinsics), c_p]),
    "sc_integrate_keyframes": (c_i32, [c_p, P(c_i32), P(c_p), P(c_p), P(Pose), c_i32, P(Intrinsics), c_p]),
    "sc_set_batch_config": (c_i32, [c_p, P(BatchConfig)]),
    "sc_get_batch_config": (c_i32, [c_p, P(BatchConfig)]),
    "sc_autotune_batch": (c_i32, [c_p, P(ReintItem), c_i32, P(Intrinsics), c_p, P(BatchConfig), P(c_f)]),
    "sc_extract_block_list": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_i32, P(c_i32), c_p]),
    "sc_marching_cubes": (c_i32, [c_p, c_p, c_p, c_i64, P(c_i64), c_p]),
    "sc_mc_case": (c_i32, [c_i32, P(c_i32)]),
    "sc_import_blocks": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_i32, c_p]),
    "sc_set_keyframe_blocks": (c_i32, [c_p, c_i32, c_p, c_i32, c_p]),
    "sc_create_block_store": (c_i32, [c_i64, c_i32, P(c_p)]),
    "sc_destroy_block_store": (c_i32, [c_p]),
    "sc_block_store_count": (c_i64, [c_p]),
    "sc_stream_out": (c_i32, [c_p, c_p, P(c_f), c_f, P(c_i64), c_p]),
    "sc_stream_in": (c_i32, [c_p, c_p, P(c_f), c_f, P(c_i64), c_p]),
    "sc_stream_in_keyframes": (c_i32, [c_p, c_p, P(c_i32), c_i32, P(c_i64), c_p]),
    "sc_stream_in_poses": (c_i32, [c_p, c_p, P(c_p), P(Pose), c_i32, P(Intrinsics), P(c_i64), c_p]),
    "sc_get_keyframe_blocks": (c_i32, [c_p, c_i32, c_p, c_i32, P(c_i32), c_p]),
    "sc_sdf_loss": (c_i32, [c_p, c_p, c_i64, c_f, c_p, c_p, c_p]),
    "sc_sdf_adjoint": (c_i32, [c_p, P(c_i32), P(c_p), P(Pose), c_i32, P(Intrinsics), c_p, c_p, c_p, c_p]),
    "sc_sdf_adjoint_noalloc": (c_i32, [c_p, P(c_i32), P(c_p), P(Pose), c_i32, P(Intrinsics), c_p, c_p, c_p, c_p]),
    "sc_pose_distance": (c_d, [P(Pose), P(Pose)]),
    "sc_select_topm": (c_i32, [P(c_d), c_i32, c_i32, P(c_i32)]),
    "sc_select_consecutive": (c_i32, [P(c_d), c_i32, c_i32]),
    "sc_pose_exp_left": (c_i32, [P(Pose), P(c_d), P(Pose)]),
    "sc_set_retry_limit": (c_i32, [c_p, c_i32]),
    "sc_abi_version": (c_i32, []),
    "sc_kernel_launches": (c_u64, []),
    "sc_measure_fp32_rate": (c_i32, [c_i32, P(c_d), P(c_d), c_p]),
    "sc_set_profiling": (c_i32, [c_p, c_i32]),
    "sc_fusion_profile": (c_i32, [c_i32, P(c_d), P(c_i64), P(c_i64)]),
    "sc_get_profile": (c_i32, [c_p, P(Profile)]),
}

_lib = None


def lib():
    """Load libsurfcorr.so (once).  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1709_03763_b300.build` "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SurfcorrError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        msg = lib().sc_status_string(self.code).decode()
        super().__init__(f"{where}: {msg} ({self.code})" if where else f"{msg} ({self.code})")


def check(rc: int, where: str = ""):
    if rc != SC_OK:
        raise SurfcorrError(rc, where)
