"""B300-native (sm_103a) keyframe surface correction for voxel-hashed TSDF reconstruction.

Implements the GPU hot path of on-the-fly surface correction (Maier, Schaller,
Cremers, arXiv 1709.03763): keyframe depth fusion (Eq. 1), block allocation in a
voxel-hashed SDF, running-average integration, de-integration (Eq. 2) and
batched re-integration on pose-graph updates (Section 4.3), plus an adjoint pass
for a loss on the fused SDF.  All compute is in libsurfcorr.so (C ABI in
include/surfcorr.h); this package marshals torch tensors into it.
"""
from ._lib import SurfcorrError, lib  # noqa: F401
from .volume import (BlockStore, Volume, depth_from_u16, rgba_from_rgb, fuse_colour_keyframes, fuse_frames_into_keyframe, fuse_keyframes, prepare_colour, make_intrinsics, prepare_fuse, make_pose, pose_distance,  # noqa: F401
                     KF_CONST, KF_DIST, KF_OVRLP, mc_case, overlap_counts, pose_exp_left, segment_keyframes,
                     select_consecutive, select_topm)
