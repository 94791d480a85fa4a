/*
 * surfcorr.h -- C ABI of the B300 (sm_103a) keyframe surface-correction library.
 *
 * The library implements the GPU hot path of on-the-fly surface correction for
 * large-scale RGB-D reconstruction (Maier, Schaller, Cremers, arXiv 1709.03763):
 * keyframe depth fusion (Eq. 1), a voxel-hashed sparse truncated SDF with
 * 8^3-voxel blocks (Section 3 "SDF volume"), keyframe integration by a running
 * weighted average, its exact inverse (de-integration, Eq. 2) and batched
 * re-integration on pose-graph updates (Section 4.3).  It adds two extensions
 * the paper does not have: one persistent, graph-captured launch per pose update
 * and an adjoint (backward) pass for a loss on the fused SDF.
 *
 * Conventions (Section 3 "Preliminaries"):
 *   - A pose is world_from_camera: p_world = R p_cam + t, stored as a row-major
 *     3x4 float matrix [R | t] (sc_pose).
 *   - Pinhole intrinsics; pixel centres at integer (u, v); pi^-1(x, Z) =
 *     ((u - cx) / fx * Z, (v - cy) / fy * Z, Z).  Depth is z-depth in metres, 0 or
 *     negative = invalid.  Images are row-major [height][width]; colour is RGBA8
 *     [height][width][4] (alpha ignored).
 *   - Voxel index i (int3) sits at world position i * voxel_size; block b holds
 *     voxels 8b .. 8b+7 on each axis.
 *
 * Memory and execution:
 *   - Image, pose-output and gradient buffers are caller-owned device memory
 *     (plain pointers, e.g. torch tensors' data_ptr()).  Device pointers must be
 *     16-byte aligned.  Pose and item arrays are host memory unless stated.
 *   - The volume (hash table, voxel pool, per-keyframe block lists, scratch)
 *     is owned by the library and allocated on the device that is current when
 *     sc_create_volume is called; every later call on that volume must run with
 *     that device current.
 *   - Calls are asynchronous on the given stream (NULL = legacy default stream)
 *     unless stated.  Calls on one volume must be serialised by the caller (one
 *     stream, or events between streams).
 *   - Device-side failures (full hash table, full pool, full block list, a
 *     bounded retry giving up) set a sticky per-volume status word; calls that
 *     synchronise return it, and sc_get_status reads and clears it.  Host-side
 *     argument errors are returned before anything is launched.
 *
 * Every entry point returns SC_OK (0) or a negative sc_status.
 */
#ifndef SURFCORR_H
#define SURFCORR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SC_ABI_VERSION 1

typedef enum {
    SC_OK = 0,
    SC_ERR_INVALID_ARG = -1,        /* bad pointer / size / id, rejected before launch */
    SC_ERR_CUDA = -2,               /* a CUDA runtime call failed */
    SC_ERR_HASH_FULL = -3,          /* no free hash entry within the probe limit */
    SC_ERR_POOL_FULL = -4,          /* voxel pool has no free block */
    SC_ERR_RETRY_LIMIT = -5,        /* a bounded device wait gave up */
    SC_ERR_NOT_INTEGRATED = -6,     /* de-integrating a keyframe id that is not integrated */
    SC_ERR_CAPACITY = -7,           /* output buffer too small (count still reported) */
    SC_ERR_ALREADY_INTEGRATED = -8, /* integrating a keyframe id that is integrated */
    SC_ERR_LIST_FULL = -9,          /* a keyframe touched more blocks than its list holds */
    SC_ERR_NOT_RESIDENT = -10,      /* a keyframe's block is in the host block store, not on the GPU */
    SC_ERR_CONFLICT = -11           /* a block streamed in is already resident on the GPU */
} sc_status;

typedef enum { SC_RGBA8 = 0, SC_RGB_F32 = 1 } sc_colour_format;

typedef void* sc_stream; /* a cudaStream_t */

typedef struct sc_volume sc_volume;

typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} sc_intrinsics;

typedef struct {
    float m[3][4]; /* [R | t], world_from_camera */
} sc_pose;

typedef struct {
    float voxel_size;                 /* metres */
    float trunc;                      /* truncation mu, metres */
    uint32_t n_buckets;               /* hash buckets, power of two */
    uint32_t bucket_size;             /* entries per bucket, 1..16 */
    uint32_t max_blocks;              /* voxel pool capacity, 8^3 blocks, <= 2^23 */
    int32_t colour_format;            /* SC_RGBA8 or SC_RGB_F32 */
    int32_t max_keyframes;            /* keyframe ids are 0 .. max_keyframes-1 */
    uint32_t max_blocks_per_keyframe; /* touched-list capacity per keyframe */
    int32_t max_batch;                /* max items per sc_reintegrate_batch (<= 1024) */
} sc_volume_params;

typedef struct {
    float disc_rel; /* drop pixels whose 4-neighbour depth differs by more than disc_rel * Z */
} sc_fusion_params;

typedef struct {
    float disc_rel; /* keyframe normal: Z* neighbours must lie within disc_rel * Z* (as in Eq. 1) */
    float occl_rel; /* a sample is visible if the frame's depth at its nearest pixel is within occl_rel * z */
} sc_colour_params;

/* One keyframe of a pose-graph update: de-integrate at old_pose, re-integrate at new_pose. */
typedef struct {
    const float* depth;   /* device [H][W] keyframe depth (same as at its integration) */
    const uint8_t* rgba;  /* device [H][W][4] keyframe colour */
    sc_pose old_pose;     /* pose it is currently integrated with */
    sc_pose new_pose;     /* updated pose */
    int32_t kf_id;
} sc_reint_item;

/* Launch configuration of the batched re-integration (chosen by sc_autotune_batch). */
typedef struct {
    int32_t warps_per_cta;   /* 2, 4, 8 or 16 */
    int32_t ctas_per_sm;     /* persistent CTAs per SM, 1..16 */
    int32_t blocks_per_grab; /* voxel blocks a warp takes from the queue at once, 1..16 */
} sc_batch_config;

typedef struct {
    uint32_t allocated_blocks; /* pool slots in use */
    uint32_t max_blocks;
    uint32_t hash_entries;     /* n_buckets * bucket_size */
    int32_t integrated_keyframes;
    uint64_t device_bytes;     /* device memory owned by the volume */
} sc_volume_info;

/* ---------------------------------------------------------------- volume ---- */

/* Create an empty volume (Section 3 "SDF volume") on the current device.
 * The hash table, voxel pool, block lists and counters are allocated here.  Other
 * calls allocate too (and can return SC_ERR_CUDA when that fails):
 *   - the first sc_reintegrate_batch / sc_integrate_keyframes / sc_autotune_batch
 *     on a volume: the batch masks, union list and item tables; the packed
 *     keyframe images again whenever the image size changes;
 *   - sc_autotune_batch: a snapshot of the volume's used blocks, freed on return;
 *   - the first sc_sdf_adjoint on a volume (and one with more keyframes than
 *     before, at least 256): its item tables and accumulators;
 *   - sc_fuse_frames_into_keyframe / sc_fuse_keyframes: 8 bytes per keyframe
 *     pixel of stream-ordered scratch per call, from a memory pool per device that
 *     keeps its memory (so only the first call, or a larger one, reaches the driver);
 *   - sc_overlap_counts (a stream-ordered count buffer per call),
 *     sc_segment_keyframes with KF_OVRLP (stream-ordered pose and group buffers per
 *     call; the first call on a device its grouping graph and state),
 *     sc_stream_in_keyframes (a stream-ordered flag array per call),
 *     sc_create_block_store, and the first sc_marching_cubes on a device (its
 *     case table).
 * sc_sdf_adjoint_noalloc allocates nothing.  Colour fusion uses a caller-owned
 * workspace.  Returns SC_ERR_INVALID_ARG for a zero or non-power-of-two bucket
 * count, a non-positive voxel size or truncation, or sizes out of range;
 * SC_ERR_CUDA if allocation fails. */
int sc_create_volume(const sc_volume_params* params, sc_volume** out);

/* Free a volume and all its device memory (synchronises the device). */
int sc_destroy_volume(sc_volume* vol);

/* Empty the volume: clear the hash table, the pool counter and every keyframe's
 * block list (stream-ordered).  Pool memory is re-initialised lazily: a block is
 * zeroed by the first update that touches it after its allocation. */
int sc_reset_volume(sc_volume* vol, sc_stream stream);

/* Read (and clear) the sticky device status word; synchronises the stream the
 * volume last used.  *device_status receives the sc_status the device reported. */
int sc_get_status(sc_volume* vol, int32_t* device_status);

int sc_get_volume_info(sc_volume* vol, sc_volume_info* info); /* synchronises */

const char* sc_status_string(int status);

/* -------------------------------------------------------- keyframe fusion ---- */

/* Eq. 1 (Section 3 "Keyframe Fusion"): warp every valid pixel x of each of the
 * n frames into the keyframe, p* = g(T*^-1, g(T_i, pi^-1(x, Z_i(x)))), round
 * pi(p*) to the nearest pixel x*, and accumulate the depth-weighted average
 *   Z*(x*) = sum w_z Z*_p / sum w_z,   W*(x*) = sum w_z,
 * with w_z = cos(theta) / Z^2 (theta: angle between the central-difference depth
 * normal and the camera axis).  Pixels on the border, with an invalid 4-neighbour
 * or a neighbour depth jump above disc_rel * Z are dropped.
 *   depths     device [n][H][W] frame depth
 *   frame_poses host [n] frame poses T_i;  kf_pose host keyframe pose T*
 *   kf_depth   device [H][W] output Z* (0 where W* = 0)
 *   kf_weight  device [H][W] output W*
 * Both outputs are overwritten.  n >= 1. */
int sc_fuse_frames_into_keyframe(const float* depths, const sc_pose* frame_poses, int32_t n,
                                 const sc_pose* kf_pose, const sc_intrinsics* intr,
                                 const sc_fusion_params* fusion, float* kf_depth, float* kf_weight,
                                 sc_stream stream);

/* Eq. 1 for many keyframes in one call: frame f (device depths [n_frames][H][W],
 * host pose frame_poses[f]) is fused into keyframe frame_kf[f] (host, 0 <= frame_kf[f]
 * < n_kf) at pose kf_poses[frame_kf[f]] (host [n_kf]).  Outputs kf_depth and
 * kf_weight are device [n_kf][H][W], overwritten.  Same per-keyframe result as
 * sc_fuse_frames_into_keyframe on each keyframe's frames (up to float summation
 * order).  Widths a multiple of 4: one launch initialises each keyframe's sums from
 * its first frame at the keyframe pose (no zeroing), then one scatter launch per 576
 * other frames and one normalisation launch; other widths zero the sums and scatter
 * every frame. */
int sc_fuse_keyframes(const float* depths, const sc_pose* frame_poses, const int32_t* frame_kf, int32_t n_frames,
                      const sc_pose* kf_poses, int32_t n_kf, const sc_intrinsics* intr,
                      const sc_fusion_params* fusion, float* kf_depth, float* kf_weight, sc_stream stream);

/* Raw sensor depth to metres: depth[i] = raw[i] * scale (one float multiply, round
 * to nearest; raw 0 gives 0, the invalid depth), for 16-bit depth images such as
 * those of Kinect-class sensors (scale 1/1000 for millimetres, 1/5000 for the TUM
 * RGB-D format).  raw and depth device [n], 16-byte aligned.  Asynchronous. */
int sc_depth_from_u16(const uint16_t* raw, int64_t n, float scale, float* depth, sc_stream stream);

/* Packed 8-bit RGB (3 bytes a pixel, the usual colour-sensor format) to the RGBA8
 * layout the volume reads: rgba[4i .. 4i+2] = rgb[3i .. 3i+2], rgba[4i+3] = 255.
 * Sending colour as RGB moves a quarter fewer bytes over the host link.  rgb device
 * [n_pixels][3], 4-byte aligned; rgba device [n_pixels][4], 16-byte aligned; the two
 * must not overlap.  n_pixels >= 0.  Asynchronous. */
int sc_rgba_from_rgb(const uint8_t* rgb, int64_t n_pixels, uint8_t* rgba, sc_stream stream);

/* ------------------------------------------------- colour keyframe fusion ---- */

/* Device workspace sc_fuse_colour_keyframes needs for width x height images:
 * 64 frames of 8-byte unsharp texels plus the blurriness sums.  0 for sizes out of
 * range (width or height < 2 or > 16384). */
uint64_t sc_colour_workspace_bytes(int32_t width, int32_t height);

/* Colour keyframe fusion (Section 3 "Keyframe Fusion", colour paragraph) for many
 * keyframes in one call.  Frame f (colour rgba, depth depths, pose frame_poses[f])
 * belongs to keyframe frame_kf[f] (depth Z* in kf_depth, pose kf_poses[...]).
 *  1. each frame's colour is deblurred by unsharp masking, S = I + (I - G*I) with G
 *     the 5x5 binomial (1 4 6 4 1)/16 per axis, borders replicated, clamped to
 *     [0, 255] (computed exactly, in 1/256 units);
 *  2. each frame gets w_b = 1 - b, b the Crete-Roffet blurriness of its luma
 *     Y = (77 R + 150 G + 29 B) / 256: per direction, with a 9-tap box mean B,
 *     b_e = (sum|dY| - sum max(0, |dY| - |dB|)) / sum|dY| (0 if sum|dY| = 0),
 *     b = max of the two directions;
 *  3. each keyframe pixel x* with Z*(x*) > 0 and a valid Eq. 1 normal (4-neighbours
 *     valid and within disc_rel * Z*; border pixels have none) is warped into every
 *     frame of its group, p_i = g(T_i^-1, g(T*, pi^-1(x*, Z*(x*)))).  A sample is
 *     kept if z_i > 0, pi(p_i) lies in [0, W-1] x [0, H-1], and the frame's depth at
 *     the nearest pixel (halves up) is > 0 and within occl_rel * z_i of z_i.  Its
 *     value is the bilinear sample of S, its weight w_c = w_b cos(theta) / z_i^2
 *     (theta between the normal, rotated into frame i, and its optical axis);
 *  4. C*(x*) per channel is the lower weighted median: the smallest sample value m
 *     with sum of the weights of samples <= m at least half the total weight;
 *     output (round(m_R), round(m_G), round(m_B), 255), halves up, or (0, 0, 0, 0)
 *     without samples.
 * rgba device [n_frames][H][W][4]; depths device [n_frames][H][W]; frame_poses and
 * frame_kf host [n_frames] (0 <= frame_kf[f] < n_kf, at most 64 frames per
 * keyframe); kf_depth device [n_kf][H][W]; kf_poses host [n_kf]; workspace device,
 * 256-byte aligned, at least sc_colour_workspace_bytes(W, H) bytes (SC_ERR_CAPACITY
 * otherwise), owned by the caller and not shared with a call that may overlap on the
 * GPU.  Outputs (device, overwritten): kf_rgba [n_kf][H][W][4]; kf_colour
 * [n_kf][H][W][3] float medians before rounding, or NULL; frame_weight [n_frames]
 * w_b, or NULL.  Device images 16-byte aligned.  Two launches per chunk of whole
 * keyframe groups of at most 64 frames. */
int sc_fuse_colour_keyframes(const uint8_t* rgba, const float* depths, const sc_pose* frame_poses,
                             const int32_t* frame_kf, int32_t n_frames, const float* kf_depth,
                             const sc_pose* kf_poses, int32_t n_kf, const sc_intrinsics* intr,
                             const sc_colour_params* params, void* workspace, uint64_t workspace_bytes,
                             uint8_t* kf_rgba, float* kf_colour, float* frame_weight, sc_stream stream);

/* ------------------------------------------------- keyframe strategies ---- */

/* Keyframe strategies (Section 4.2). */
typedef enum {
    SC_KF_CONST = 0, /* params[0] = kappa: a new keyframe every kappa frames */
    SC_KF_DIST = 1,  /* params[0] = thr_t (m), params[1] = thr_r (rad): a new keyframe when the
                        current frame's pose is more than thr_t away from the current keyframe's
                        (|t_f - t_k|) or rotated by more than thr_r (angle of R_k^T R_f) */
    SC_KF_OVRLP = 2  /* params[0] = thr in [0, 1]: a new keyframe when the overlap ratio of the
                        current frame with the current keyframe (sc_overlap_counts) < thr */
} sc_kf_strategy;

/* Overlap of frames with a keyframe (KF_OVRLP, Section 4.2): for each frame i, counts
 * (device, out [n][2] uint64) = (valid pixels Z > 0, valid pixels whose point, warped
 * with pi^-1, the frame pose and the keyframe pose, is in front of the keyframe and
 * has its nearest pixel (halves up) inside the keyframe image).  The overlap ratio is
 * counts[i][1] / counts[i][0].  depths device [n][H][W]; poses host.  Asynchronous. */
int sc_overlap_counts(const float* depths, const sc_pose* frame_poses, int32_t n, const sc_pose* kf_pose,
                      const sc_intrinsics* intr, uint64_t* counts, sc_stream stream);

/* Group frames 0..n-1 (in order) into keyframes: frame 0 starts the first group, a frame
 * that meets the strategy's condition against the current keyframe starts the next
 * group and becomes its keyframe (its pose is the keyframe pose).  frame_kf (host, out
 * [n]) receives each frame's group, *n_keyframes their number.  depths (device
 * [n][H][W]) and intr are needed for SC_KF_OVRLP only (otherwise may be NULL).  KF_DIST
 * distances are computed in double from the float poses; KF_OVRLP ratios from integer
 * counts.  KF_OVRLP runs its grouping loop on the device (a CUDA graph with a while
 * node: per step, the overlap counts of the next 8 to 32 frames and one decision
 * kernel), then reads the groups back and synchronises the stream once.  The first
 * KF_OVRLP call on a device, and the first with a new image size, builds that graph
 * (it and its state stay allocated until exit); concurrent KF_OVRLP calls on one
 * device take turns. */
int sc_segment_keyframes(int32_t strategy, const double* params, const float* depths, const sc_pose* poses,
                         int32_t n, const sc_intrinsics* intr, int32_t* frame_kf, int32_t* n_keyframes,
                         sc_stream stream);

/* ------------------------------------------------ integration (plain path) ---- */

/* Integrate keyframe kf_id at pose T (Section 3 "SDF volume": voxel blocks are
 * first allocated, then updated with a running weighted average):
 *  1. allocation: every block whose closed box meets the band segment
 *     {pi^-1(x, z) : z in [Z(x) - mu, Z(x) + mu]} (world coordinates) of a valid
 *     pixel x is inserted into the hash table if absent; the set of these blocks,
 *     A(k, T), becomes the keyframe's block list;
 *  2. update: for each voxel v of each block in A(k, T): p_c = R^T (p_v - t);
 *     x = nearest pixel of pi(p_c) (halves up); if z_c > 0, x inside the image,
 *     Z(x) > 0 and eta = Z(x) - z_c >= -mu:
 *       d = min(eta, mu), w = 1, c = rgba(x).rgb,
 *       D <- (D W + d w) / (W + w),  C <- (C W + c w) / (W + w),  W <- W + w.
 * depth device [H][W]; rgba device [H][W][4]; pose host.
 * Returns SC_ERR_ALREADY_INTEGRATED if kf_id is integrated. */
int sc_integrate_keyframe(sc_volume* vol, int32_t kf_id, const float* depth, const uint8_t* rgba,
                          const sc_intrinsics* intr, const sc_pose* pose, sc_stream stream);

/* De-integrate keyframe kf_id (Eq. 2, Section 4.3): over the keyframe's stored
 * block list, with the same per-voxel d, c, w as its integration,
 *   D <- (D W - d w) / (W - w),  C <- (C W - c w) / (W - w),  W <- W - w,
 * and D = C = 0 where W reaches 0.  depth, rgba and pose must be the ones kf_id
 * was integrated with.  Returns SC_ERR_NOT_INTEGRATED if kf_id is not integrated. */
int sc_deintegrate_keyframe(sc_volume* vol, int32_t kf_id, const float* depth, const uint8_t* rgba,
                            const sc_intrinsics* intr, const sc_pose* pose, sc_stream stream);

/* ------------------------------------------------ batched re-integration ---- */

/* One pose-graph update (Section 4.3 "Re-integration strategy"): de-integrate
 * every item at old_pose and re-integrate it at new_pose.  The result equals
 * de-integrating all items in order and then integrating all items in order
 * (up to float rounding): the new poses' blocks are allocated first, then every
 * voxel touched by any item receives its summed net change in one
 * read-modify-write.  Runs as one CUDA graph (replayed across calls) whose voxel
 * work is a single persistent launch.  items host [n], 1 <= n <= max_batch, kf_ids
 * distinct and integrated.  Asynchronous: argument errors return at once; device
 * errors (full hash table, pool or block list) set the sticky status word that
 * sc_get_status and the synchronising calls report, after which the volume's contents
 * are undefined.  The call waits only until the launch two batch calls back has read
 * its item table (two alternating host staging copies); with profiling on
 * (sc_set_profiling) it synchronises and returns the device status.  The batch packs
 * each item's depth and colour into one texel image per position in the batch; an
 * item whose keyframe the previous batch packed at the same position from the same
 * pointers, and which has stayed integrated since, is not packed again (an integrated
 * keyframe's images must not change: its de-integration needs them). */
int sc_reintegrate_batch(sc_volume* vol, const sc_reint_item* items, int32_t n, const sc_intrinsics* intr,
                         sc_stream stream);

/* Integrate n keyframes that are not integrated yet (Section 3 "SDF volume") in
 * one graph launch: the allocation of every keyframe's blocks, then one
 * read-modify-write per touched voxel with the keyframes' summed contributions.
 * Equal to n sc_integrate_keyframe calls in order, up to float summation order.
 * kf_ids, depths (device pointers), rgbas (device pointers), poses: host [n],
 * 1 <= n <= max_batch, ids distinct.  Asynchronous, as sc_reintegrate_batch. */
int sc_integrate_keyframes(sc_volume* vol, const int32_t* kf_ids, const float* const* depths,
                           const uint8_t* const* rgbas, const sc_pose* poses, int32_t n, const sc_intrinsics* intr,
                           sc_stream stream);

/* Set / read the launch configuration of sc_reintegrate_batch. */
int sc_set_batch_config(sc_volume* vol, const sc_batch_config* cfg);
int sc_get_batch_config(sc_volume* vol, sc_batch_config* cfg);

/* Time each candidate configuration on this batch and keep the fastest.  The
 * volume is snapshotted before and restored after every trial, so on return it
 * is unchanged; the batch itself is NOT applied.  ms_out (host, may be NULL)
 * receives the best time per batch.  Synchronises; needs device memory for one
 * snapshot of the used pool. */
int sc_autotune_batch(sc_volume* vol, const sc_reint_item* items, int32_t n, const sc_intrinsics* intr,
                      sc_stream stream, sc_batch_config* best, float* ms_out);

/* ------------------------------------------------------------ extraction ---- */

/* Compact the occupied hash entries (Section 3: extraction of the allocated
 * blocks precedes surface extraction) into block coordinates coords [cap][3] and
 * pool slots slots [cap] (device, either may be NULL).  If D, W or C are given
 * (device [cap][512] float, [cap][512] float, and [cap][512][4] uint8 for RGBA8 or
 * [cap][512][3] float for RGB_F32, voxel index x + 8y + 64z), the voxel payloads
 * are copied too.  Block order is unspecified.  *count (host) receives the number
 * of blocks; SC_ERR_CAPACITY if it exceeds capacity (the first capacity blocks
 * are written).  Synchronises. */
int sc_extract_block_list(sc_volume* vol, int32_t* coords, int32_t* slots, float* D, float* W, void* C,
                          int32_t capacity, int32_t* count, sc_stream stream);

/* Copy the block list stored for kf_id (pool slots, device out [capacity]) and
 * its length (*count, host).  Synchronises. */
int sc_get_keyframe_blocks(sc_volume* vol, int32_t kf_id, int32_t* slots, int32_t capacity, int32_t* count,
                           sc_stream stream);

/* ------------------------------------------------- marching cubes, import ---- */

/* Iso-surface extraction (Section 3 "SDF volume": the surface is extracted with
 * Marching Cubes).  Cube (x, y, z) has the corner voxels (x + i0, y + i1, z + i2),
 * i0..i2 the bits of the corner number 0..7; it is meshed when all 8 corner voxels
 * are allocated and observed (W > 0).  A corner is inside when D < 0; each cube
 * edge between an inside and an outside corner carries the vertex
 * p = voxel_size * (v_lo + t e_axis), t = D_lo / (D_lo - D_hi).  Edge e (0..11)
 * runs along axis e / 4 from the corner whose two other coordinate bits are e % 4
 * (lower axis in bit 0).  Triangulation rule: on each cube face, every maximal run
 * of inside corners around the face (not all four) is closed off by one segment
 * joining the crossed edges at its ends (diagonal inside corners are cut off
 * separately); the segments chain into loops oriented so that triangle normals
 * (v1 - v0) x (v2 - v0) point to D > 0; each loop is fanned from its smallest edge,
 * loops in order of their smallest edge.  At most 5 triangles per cube.
 * triangles device [capacity][3][3] float (metres, world frame of the volume);
 * cubes device [capacity][4] int32 (first corner voxel x, y, z and the triangle's
 * number within its cube) or NULL.  *count (host) receives the number of
 * triangles; output order is unspecified; SC_ERR_CAPACITY if it exceeds capacity
 * (the first `capacity` found are written).  Synchronises the stream. */
int sc_marching_cubes(sc_volume* vol, float* triangles, int32_t* cubes, int64_t capacity, int64_t* count,
                      sc_stream stream);

/* The triangulation rule alone: for the inside-corner mask (0..255), writes the
 * edge triples of its triangles to edges (host, up to 15 ints) and returns their
 * number (0..5), or a negative status.  Host only. */
int sc_mc_case(int32_t mask, int32_t* edges);

/* Load voxel blocks into a volume (restore, or a volume made elsewhere): for each of
 * n blocks, coords device [n][3] int32 block coordinates (distinct, each in
 * [-2^20, 2^20)), D and W device [n][512] float (voxel x + 8 y + 64 z), C device
 * [n][512] uint32 RGBA8 or [n][3][512] float (the volume's colour format) or NULL
 * (black).  An absent block is inserted and takes a pool slot; a present one is
 * overwritten.  Keyframe block lists are not changed.  Device arrays 16-byte
 * aligned.  Returns SC_ERR_INVALID_ARG for a coordinate out of range, SC_ERR_HASH_FULL
 * / SC_ERR_POOL_FULL when the volume is full.  Synchronises the stream. */
int sc_import_blocks(sc_volume* vol, const int32_t* coords, const float* D, const float* W, const void* C,
                     int32_t n, sc_stream stream);

/* Restore a keyframe's block list A(k, T) (checkpoint / resume): coords device [n][3]
 * int32, the block coordinates of its list (e.g. sc_get_keyframe_blocks mapped to
 * coordinates before the checkpoint), all resident in the volume.  Marks kf_id
 * integrated, so that it can be de-integrated and re-integrated with the depth,
 * colour and pose it was integrated with.  SC_ERR_ALREADY_INTEGRATED if kf_id is
 * integrated, SC_ERR_LIST_FULL if n > max_blocks_per_keyframe, SC_ERR_INVALID_ARG
 * (kf_id left not integrated) if a coordinate has no resident block.  Synchronises. */
int sc_set_keyframe_blocks(sc_volume* vol, int32_t kf_id, const int32_t* coords, int32_t n, sc_stream stream);

/* -------------------------------------------------- the streaming sphere ---- */

/* Host block store of the streaming sphere (Section 3 "SDF volume": only blocks within
 * a sphere of constant radius around the camera stay in GPU memory; the others are
 * streamed to the host).  Pinned, device-mapped host memory for `capacity` blocks
 * (12 KB each in RGBA8, 20 KB in RGB_F32) on the current device; colour_format must
 * match the volumes it serves. */
typedef struct sc_block_store sc_block_store;
int sc_create_block_store(int64_t capacity, int32_t colour_format, sc_block_store** out);
int sc_destroy_block_store(sc_block_store* store);
/* Blocks held by the store (-1 for NULL). */
int64_t sc_block_store_count(const sc_block_store* store);

/* Stream out: every resident block whose centre ((8 b + 3.5) * voxel_size per axis) is
 * farther than `radius` from `centre` (host float[3], metres; distance compared
 * squared in float) moves into the store with its D, W, C and initialisation flag.
 * The pool is compacted (the remaining blocks keep their data, some change slot), the
 * hash table is rebuilt, and keyframe block lists keep naming every block of their
 * A(k, T): resident blocks by slot, stored ones by an external id.  De-integrating,
 * re-integrating (sc_reintegrate_batch) or differentiating (sc_sdf_adjoint) a
 * keyframe whose list names a stored block returns SC_ERR_NOT_RESIDENT before any
 * launch; stream those blocks in first.  Integrating a new keyframe over a region
 * whose blocks are stored allocates fresh blocks there and makes their later
 * stream-in fail with SC_ERR_CONFLICT, so stream a region in before integrating
 * into it (the paper streams the sphere around the camera before each
 * integration).  *n_moved (host) = blocks moved.  SC_ERR_CAPACITY if the store
 * cannot take them (nothing moves).  Synchronises the stream. */
int sc_stream_out(sc_volume* vol, sc_block_store* store, const float* centre, float radius, int64_t* n_moved,
                  sc_stream stream);

/* Stream in: every stored block whose centre is within `radius` of `centre` (the same
 * test) returns to the GPU at a new pool slot, and list entries naming it become its
 * slot.  A stored block whose coordinate has been allocated on the GPU meanwhile
 * stays stored and the call returns SC_ERR_CONFLICT (stream in before integrating
 * into a region).  radius = +inf streams in everything.  Synchronises the stream. */
int sc_stream_in(sc_volume* vol, sc_block_store* store, const float* centre, float radius, int64_t* n_moved,
                 sc_stream stream);

/* Stream in exactly the stored blocks that the current block lists of keyframes
 * kf_ids (host [n]) name, so that those keyframes can be de-/re-integrated (the
 * paper streams in the sphere around T_j* "to safely access them"; this streams the
 * blocks the keyframes need, each once).  Same rules and errors as sc_stream_in.
 * Synchronises the stream. */
int sc_stream_in_keyframes(sc_volume* vol, sc_block_store* store, const int32_t* kf_ids, int32_t n,
                           int64_t* n_moved, sc_stream stream);

/* Stream in exactly the stored blocks that allocating A(k, T) (Section 3 "SDF
 * volume") for n keyframe images at the given poses would reach: the allocation's own
 * walk of every valid pixel's band segment, each block looked up in the store's key
 * index.  Called before re-integrating keyframes at updated poses (Section 4.3 streams
 * the spheres around the updated poses in; this streams in the blocks the new poses'
 * allocation needs, each once), so that the allocation finds them resident instead of
 * creating second copies.
 *   depths  host [n] array of device [H][W] keyframe depth pointers
 *   poses   host [n] updated poses;  intr: the images' intrinsics
 * Same rules and errors as sc_stream_in; n = 0 moves nothing.  Synchronises. */
int sc_stream_in_poses(sc_volume* vol, sc_block_store* store, const float* const* depths, const sc_pose* poses,
                       int32_t n, const sc_intrinsics* intr, int64_t* n_moved, sc_stream stream);

/* --------------------------------------------- loss and adjoint (extension) ---- */

/* Loss on the fused SDF (no counterpart in the paper):
 *   L = (1/P) sum_p Dt(p)^2 + lambda * sum_v W D^2 / sum_v W,
 * Dt the trilinear interpolation of D over the 8 voxels around point p (voxel i
 * at i * voxel_size); points whose 8 voxels are not all observed (W > 0) are
 * dropped; P counts the rest.  Writes dL/dD for every voxel of the allocated
 * pool slots [0, allocated_blocks) into grad_D (device [max_blocks][512] float;
 * entries of unallocated slots are left untouched) and, into out (device, 5
 * doubles), {L, P, sum_p Dt^2, sum_v W D^2, sum_v W}.  points device [n][3]
 * float. */
int sc_sdf_loss(sc_volume* vol, const float* points, int64_t n, float lambda, float* grad_D, double* out,
                sc_stream stream);

/* Adjoint of the keyframe integrations: given dL/dD (grad_D, from sc_sdf_loss),
 * the gradient of L with respect to each keyframe's pose (left se(3)
 * perturbation exp(xi^) T, xi = (rho, omega), at xi = 0) and depth pixels.
 * Uses D(v) = sum_k w_k d_k(v) / W(v) and recomputes each voxel's projection:
 * for each voxel of the keyframe's block list that its integration updated
 * without clamping (eta < mu), g = dL/dD(v) w / W(v) contributes
 *   dL/dZ_k(x) += g,   dL/drho += g r3,   dL/domega += g (p_v x r3),
 * r3 = R e3 (camera z axis in world coordinates).  Discrete decisions (pixel,
 * band, clamp) contribute nothing.
 *   kf_ids, poses  host [n]; depths host [n] array of device [H][W] pointers
 *   grad_xi        device [n][6] double, overwritten
 *   grad_depth     device [n][H][W] float or NULL, overwritten
 * Its keyframe tables and accumulators belong to the volume (allocated by the
 * first call, grown when n exceeds them), so calls on different volumes share no
 * scratch.  Asynchronous: before it rewrites the tables the call waits only until the
 * previous call's copies of them have been made (not for other queued work). */
int sc_sdf_adjoint(sc_volume* vol, const int32_t* kf_ids, const float* const* depths, const sc_pose* poses,
                   int32_t n, const sc_intrinsics* intr, const float* grad_D, double* grad_xi, float* grad_depth,
                   sc_stream stream);

/* sc_sdf_adjoint without any device-memory allocation by the library (the paper has
 * no counterpart; this is a deployment variant).  For callers that cannot call
 * cudaMalloc once running -- a real-time thread with a memory budget fixed at
 * start-up, an application whose device memory belongs to another allocator.  Same
 * arguments and results as sc_sdf_adjoint (the caller still passes grad_D, grad_xi
 * and grad_depth); its keyframe table and accumulators live in a file-scope device
 * array of about 76 KB that every GPU loading the library holds until the process
 * exits.
 *   - n <= 256 keyframes; more returns SC_ERR_CAPACITY and launches nothing.
 *   - The volume's device must be the current device (else SC_ERR_INVALID_ARG).
 *   - The first call on a device looks up the array's device address (with that
 *     device current; concurrent first calls are serialised by a lock); make that
 *     first call before any stream capture.
 *   - All calls share the array: calls whose work overlaps on the GPU (other
 *     streams, other host threads, other volumes on the same device) race and give
 *     wrong results; serialise them.  Each call clears the accumulators it uses. */
int sc_sdf_adjoint_noalloc(sc_volume* vol, const int32_t* kf_ids, const float* const* depths, const sc_pose* poses,
                           int32_t n, const sc_intrinsics* intr, const float* grad_D, double* grad_xi,
                           float* grad_depth, sc_stream stream);

/* ------------------------------------------------ keyframe selection (host) ---- */

/* ||s t - s t'|| (Section 4.3) with t = (Z-Y-X Euler angles of R in radians,
 * translation), s = (2,2,2,1,1,1); angle differences wrapped to (-pi, pi]. */
double sc_pose_distance(const sc_pose* a, const sc_pose* b);

/* BundleFusion's rule (Section 4.3): the m keyframes with the largest distance,
 * ties to the lower index.  dist host [K]; out host [min(m, K)]. */
int sc_select_topm(const double* dist, int32_t K, int32_t m, int32_t* out);

/* Eq. 3: first index j (0-based) of the m consecutive keyframes with the largest
 * summed distance, ties to the smallest j.  Returns j, or a negative sc_status. */
int sc_select_consecutive(const double* dist, int32_t K, int32_t m);

/* exp(xi^) T: the pose T moved by the left se(3) perturbation xi = (rho, omega)
 * (host, double precision, rounded to float once); the perturbation whose
 * gradient sc_sdf_adjoint returns. */
int sc_pose_exp_left(const sc_pose* T, const double* xi, sc_pose* out);

/* ----------------------------------------------------------------- debug ---- */

/* Per-kernel timing of the volume's own launches (CUDA events on the launching
 * stream, event nodes inside the batch graph) and the work they covered. */
typedef struct {
    int32_t enabled;
    int32_t pad;
    double alloc_ms;            /* plain-path block allocation */
    int64_t alloc_launches;
    double update_ms;           /* plain-path voxel update (integrate and de-integrate) */
    int64_t update_launches;
    int64_t update_blocks;      /* sum of the updated block-list lengths */
    double batch_alloc_ms;      /* batched allocation of the new poses' blocks */
    double batch_mark_ms;       /* marking of the old footprints */
    double batch_net_ms;        /* persistent net-delta voxel update */
    int64_t batch_launches;
    int64_t batch_union_blocks; /* sum over batches of the union of touched blocks */
    int64_t batch_pairs;        /* sum over batches of old + new block-list lengths */
    double mc_ms;               /* Marching Cubes kernel (sc_marching_cubes) */
    int64_t mc_launches;
} sc_profile;

/* Process-wide timing of the fusion launches: enable 1 / 0 resets the counters and
 * switches timing on / off, -1 only reads.  Outputs (host, may be NULL): summed
 * milliseconds, fusion launches and frames since the last reset.  Synchronises on
 * the recorded events. */
int sc_fusion_profile(int32_t enable, double* ms, int64_t* launches, int64_t* frames);

/* Enable (1) or disable (0) timing; either way the counters are reset. */
int sc_set_profiling(sc_volume* vol, int32_t enabled);
/* Read the counters (synchronises the volume's last stream). */
int sc_get_profile(sc_volume* vol, sc_profile* out);


/* Cap on every bounded device wait (slot publication, queue) in iterations; a
 * cap of 1 forces the give-up path.  0 restores the default. */
int sc_set_retry_limit(sc_volume* vol, int32_t limit);

int sc_abi_version(void);

/* Measurement support (no counterpart in the paper): the FP32 FMA rate of the
 * current device, from one full-occupancy launch in which every thread runs
 * `iters` x 32 independent-chain FMAs (after one shorter warm-up launch), timed
 * with CUDA events on `stream`.  *lane_fma_per_s receives lane FMAs per second
 * (counting FMAs only; the loop's own instructions take a few further issue
 * slots), *ms_out (may be NULL) the timed launch's milliseconds.  Synchronises;
 * writes no memory.  1 <= iters <= 2^24, else SC_ERR_INVALID_ARG. */
int sc_measure_fp32_rate(int32_t iters, double* lane_fma_per_s, double* ms_out, sc_stream stream);

/* Number of kernels this library has launched in the process so far (a graph
 * launch counts its kernel nodes). */
uint64_t sc_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SURFCORR_H */
