"""Seeded synthetic RGB-D inputs: analytic scenes, trajectories, sensor noise, pose drift.

This module only *generates inputs*.  It holds none of the surface-correction
arithmetic (fusion, allocation, TSDF update, selection, loss): it is shared by
the FP64 oracle tests and by the CUDA path, and neither of those imports the other.

The scenes stand in for the paper's RGB-D sequences (Section 5 "Datasets":
AUG_ICL/Liv1 and BundleFusion/apt0), which are not available here.  They take
those sequences' shape: 640x480 Kinect-class depth + colour at 30 fps
(Section 3 "Preliminaries"), room / apartment scale, long trajectories, and
loop-closure-style pose corrections.

Conventions
-----------
* World frame: metres, z up.
* Camera frame: x right, y down, z forward (pinhole, Section 3).
* A pose is world_from_camera, stored as a float array [3, 4] = [R | t],
  so that p_world = R p_cam + t  (the paper's g(T, p) = R p + t).
* Depth is z-depth (the z coordinate in the camera frame), 0 = invalid.
* Pixel centres sit at integer (u, v); the ray through pixel (u, v) has camera
  direction ((u - cx)/fx, (v - cy)/fy, 1).

Random streams: numpy PCG64 seeded with 1709_03763 + 1000*config + stream,
stream 0 scene, 1 trajectory, 2 noise, 3 invalid mask, 4 perturbation,
5 sample points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SEED_BASE = 1709_03763
STREAM_SCENE, STREAM_TRAJ, STREAM_NOISE, STREAM_MASK, STREAM_PERTURB, STREAM_POINTS, STREAM_BLUR = range(7)

# Depth sensor model (Kinect-class): valid range and axial noise sigma(z).
Z_MIN, Z_MAX = 0.4, 4.0
INVALID_FRACTION = 0.02


def rng(config: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * config + stream))


def noise_sigma(z):
    """Axial depth noise sigma(z) = 0.0012 + 0.0019 (z - 0.4)^2 (metres)."""
    return 0.0012 + 0.0019 * (z - 0.4) ** 2


@dataclass
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_tuple(self):
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


KINECT = Intrinsics(525.0, 525.0, 319.5, 239.5, 640, 480)
QVGA = Intrinsics(262.5, 262.5, 159.5, 119.5, 320, 240)


@dataclass
class Scene:
    """Analytic primitives.  Boxes/shell faces are ordered (-x,+x,-y,+y,-z,+z)."""
    shell: np.ndarray                      # [6] room bounds xmin,ymin,zmin,xmax,ymax,zmax (seen from inside)
    shell_colours: np.ndarray              # [6,3] uint8
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))
    box_colours: np.ndarray = field(default_factory=lambda: np.zeros((0, 6, 3), np.uint8))
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))       # cx,cy,cz,r
    sphere_colours: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.uint8))
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))     # cx,cy,r,zmin,zmax (vertical)
    cylinder_colours: np.ndarray = field(default_factory=lambda: np.zeros((0, 2, 3), np.uint8))  # side, top

    def inside_solid(self, p, margin=0.0):
        """True if point p (3,) lies inside (or within margin of) any solid primitive."""
        p = np.asarray(p, np.float64)
        for b in self.boxes:
            if np.all(p >= b[:3] - margin) and np.all(p <= b[3:] + margin):
                return True
        for s in self.spheres:
            if np.linalg.norm(p - s[:3]) <= s[3] + margin:
                return True
        for c in self.cylinders:
            if (math.hypot(p[0] - c[0], p[1] - c[1]) <= c[2] + margin
                    and c[3] - margin <= p[2] <= c[4] + margin):
                return True
        return False


# ----------------------------------------------------------------------------
# Poses
# ----------------------------------------------------------------------------

def look_pose(position, yaw, pitch, roll=0.0) -> np.ndarray:
    """world_from_camera [3,4] for a camera at `position` heading `yaw` (about world z,
    0 = +x) and tilted down by `pitch` radians (positive = looking down)."""
    fwd = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), -math.sin(pitch)])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)
    if roll != 0.0:
        R = R @ axis_angle(np.array([0.0, 0.0, 1.0]), roll)
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = position
    return T


def axis_angle(axis, angle) -> np.ndarray:
    """Rotation matrix for `angle` radians about unit `axis` (Rodrigues)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def perturb_pose(T, angle, shift, g: np.random.Generator) -> np.ndarray:
    """Left-multiply pose T by a rotation of `angle` rad about a random axis (about the
    camera centre) and a translation of `shift` m along a random direction."""
    axis = g.normal(size=3)
    d = g.normal(size=3)
    d = d / np.linalg.norm(d)
    Rp = axis_angle(axis, angle)
    out = np.array(T, np.float64).copy()
    out[:, :3] = Rp @ out[:, :3]
    out[:, 3] = out[:, 3] + shift * d
    return out


# ----------------------------------------------------------------------------
# Ray casting (z-depth at pixel centres)
# ----------------------------------------------------------------------------

def _tt(a, device, dtype):
    return torch.as_tensor(np.asarray(a), device=device, dtype=dtype)


def _slab(o, d_inv, lo, hi):
    """Per-ray slab interval against boxes: o [P,3], d_inv [P,3], lo/hi [B,3] -> tmin/tmax [P,B,3]."""
    t1 = (lo[None] - o[:, None]) * d_inv[:, None]
    t2 = (hi[None] - o[:, None]) * d_inv[:, None]
    return torch.minimum(t1, t2), torch.maximum(t1, t2)


def _near(scene: Scene, o, radius):
    """Indices of the boxes, spheres and cylinders within `radius` of point o (closest
    point of each primitive's bounding box)."""
    def box_dist(lo, hi):
        q = np.clip(o[None, :], lo, hi)
        return np.linalg.norm(q - o[None, :], axis=1)
    b = scene.boxes.reshape(-1, 6)
    sp = scene.spheres.reshape(-1, 4)
    cy = scene.cylinders.reshape(-1, 5)
    bi = np.nonzero(box_dist(b[:, :3], b[:, 3:]) <= radius)[0]
    si = np.nonzero(np.linalg.norm(sp[:, :3] - o[None, :], axis=1) - sp[:, 3] <= radius)[0]
    clo = np.stack([cy[:, 0] - cy[:, 2], cy[:, 1] - cy[:, 2], cy[:, 3]], 1)
    chi = np.stack([cy[:, 0] + cy[:, 2], cy[:, 1] + cy[:, 2], cy[:, 4]], 1)
    ci = np.nonzero(box_dist(clo, chi) <= radius)[0] if len(cy) else np.zeros(0, np.int64)
    return bi, si, ci


def render(scene: Scene, intr: Intrinsics, poses, *, device="cpu", dtype=torch.float64,
           chunk_prims: int = 64, texture: bool = False, cull_radius: float | None = None):
    """Ray-cast z-depth and colour for each pose.

    poses: [n,3,4] world_from_camera.  Returns (depth [n,H,W] float32 torch on
    `device`, rgba [n,H,W,4] uint8 torch on `device`), noise-free, 0 where no hit.
    texture=True modulates each surface colour by a smooth procedural pattern of the
    world position (the same surface point has the same colour in every view).
    cull_radius: skip primitives farther than this from the camera.  A hit at distance
    r has z-depth at least r / |(x_n, y_n, 1)| (>= r / 1.23 at 640x480, f = 525), so with
    cull_radius = 6 m every skipped hit lies beyond 4.8 m of depth, where the sensor
    model reports no depth: valid depth pixels are exactly those of a full render.
    """
    poses = np.asarray(poses, np.float64).reshape(-1, 3, 4)
    H, W = intr.height, intr.width
    vv, uu = torch.meshgrid(torch.arange(H, device=device, dtype=dtype),
                            torch.arange(W, device=device, dtype=dtype), indexing="ij")
    dcam = torch.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy,
                        torch.ones_like(uu)], dim=-1).reshape(-1, 3)
    P = dcam.shape[0]
    depth_out = torch.zeros((len(poses), H, W), device=device, dtype=torch.float32)
    rgba_out = torch.zeros((len(poses), H, W, 4), device=device, dtype=torch.uint8)

    boxes = _tt(scene.boxes.reshape(-1, 6), device, dtype)
    box_col = _tt(scene.box_colours.reshape(-1, 6, 3), device, torch.int32)
    sph = _tt(scene.spheres.reshape(-1, 4), device, dtype)
    sph_col = _tt(scene.sphere_colours.reshape(-1, 3), device, torch.int32)
    cyl = _tt(scene.cylinders.reshape(-1, 5), device, dtype)
    cyl_col = _tt(scene.cylinder_colours.reshape(-1, 2, 3), device, torch.int32)
    shell = _tt(scene.shell.reshape(6), device, dtype)
    shell_col = _tt(scene.shell_colours.reshape(6, 3), device, torch.int32)
    inf = torch.tensor(float("inf"), device=device, dtype=dtype)

    boxes_all, box_col_all, sph_all, sph_col_all, cyl_all, cyl_col_all = boxes, box_col, sph, sph_col, cyl, cyl_col
    for k, T in enumerate(poses):
        if cull_radius is not None:
            bi, si, ci = (torch.as_tensor(i, device=device, dtype=torch.long)
                          for i in _near(scene, np.asarray(T[:, 3], np.float64), cull_radius))
            boxes, box_col = boxes_all[bi], box_col_all[bi]
            sph, sph_col = sph_all[si], sph_col_all[si]
            cyl, cyl_col = cyl_all[ci], cyl_col_all[ci]
        R = _tt(T[:, :3], device, dtype)
        o = _tt(T[:, 3], device, dtype).expand(P, 3)
        d = dcam @ R.T
        # avoid exact zeros in direction components (slab test divides)
        d = torch.where(d.abs() < 1e-12, torch.full_like(d, 1e-12), d)
        d_inv = 1.0 / d
        best = torch.full((P,), float("inf"), device=device, dtype=dtype)
        col = torch.zeros((P, 3), device=device, dtype=torch.int32)

        # room shell, seen from inside: exit distance
        tmin, tmax = _slab(o, d_inv, shell[None, :3], shell[None, 3:])
        tfar, ax = tmax[:, 0].min(dim=-1)
        face = 2 * ax + (d.gather(1, ax[:, None])[:, 0] > 0).long()
        hit = tfar > 0
        best = torch.where(hit, tfar, best)
        col = torch.where(hit[:, None], shell_col[face], col)

        for s in range(0, boxes.shape[0], chunk_prims):
            bx = boxes[s:s + chunk_prims]
            tmin, tmax = _slab(o, d_inv, bx[:, :3], bx[:, 3:])
            tnear, ax = tmin.max(dim=-1)
            tfar = tmax.min(dim=-1).values
            ok = (tnear <= tfar) & (tnear > 1e-9)
            t = torch.where(ok, tnear, inf)
            tb, j = t.min(dim=1)
            axj = ax.gather(1, j[:, None])[:, 0]
            face = 2 * axj + (d.gather(1, axj[:, None])[:, 0] < 0).long()
            c = box_col[s + j, face]
            upd = tb < best
            best = torch.where(upd, tb, best)
            col = torch.where(upd[:, None], c, col)

        for s in range(0, sph.shape[0], chunk_prims):
            sp = sph[s:s + chunk_prims]
            oc = o[:, None, :] - sp[None, :, :3]
            a = (d * d).sum(-1)[:, None]
            b = 2.0 * (d[:, None, :] * oc).sum(-1)
            c0 = (oc * oc).sum(-1) - sp[None, :, 3] ** 2
            disc = b * b - 4 * a * c0
            t = (-b - torch.sqrt(disc.clamp_min(0))) / (2 * a)
            t = torch.where((disc >= 0) & (t > 1e-9), t, inf)
            tb, j = t.min(dim=1)
            upd = tb < best
            best = torch.where(upd, tb, best)
            col = torch.where(upd[:, None], sph_col[s + j], col)

        for s in range(0, cyl.shape[0], chunk_prims):
            cy = cyl[s:s + chunk_prims]
            ox = o[:, None, 0] - cy[None, :, 0]
            oy = o[:, None, 1] - cy[None, :, 1]
            dx, dy, dz = d[:, None, 0], d[:, None, 1], d[:, None, 2]
            a = dx * dx + dy * dy
            b = 2 * (dx * ox + dy * oy)
            c0 = ox * ox + oy * oy - cy[None, :, 2] ** 2
            disc = b * b - 4 * a * c0
            ts = (-b - torch.sqrt(disc.clamp_min(0))) / (2 * a)
            zs = o[:, None, 2] + ts * dz
            side_ok = (disc >= 0) & (ts > 1e-9) & (zs >= cy[None, :, 3]) & (zs <= cy[None, :, 4])
            ts = torch.where(side_ok, ts, inf)
            tt = (cy[None, :, 4] - o[:, None, 2]) / dz
            xt = ox + tt * dx
            yt = oy + tt * dy
            top_ok = (dz < 0) & (tt > 1e-9) & (xt * xt + yt * yt <= cy[None, :, 2] ** 2)
            tt = torch.where(top_ok, tt, inf)
            t = torch.minimum(ts, tt)
            tb, j = t.min(dim=1)
            is_top = tt.gather(1, j[:, None])[:, 0] < ts.gather(1, j[:, None])[:, 0]
            c = cyl_col[s + j, is_top.long()]
            upd = tb < best
            best = torch.where(upd, tb, best)
            col = torch.where(upd[:, None], c, col)

        z = torch.where(torch.isfinite(best), best, torch.zeros_like(best))
        depth_out[k] = z.reshape(H, W).to(torch.float32)
        if texture:
            p = o + z[:, None] * d
            g = texture_gain(p[:, 0], p[:, 1], p[:, 2])
            col = torch.clamp(torch.round(col.to(dtype) * g[:, None]), 0, 255).to(torch.int32)
        rgba_out[k, ..., :3] = col.reshape(H, W, 3).to(torch.uint8)
        rgba_out[k, ..., 3] = 255
    return depth_out, rgba_out


def texture_gain(x, y, z):
    """Procedural surface texture in [0.23, 1.15]: two smooth waves (periods of
    0.5-2 m) and a fine one (about 0.15 m)."""
    return 1.15 * (0.6 + 0.25 * torch.sin(9.1 * x + 4.3 * y) * torch.cos(7.7 * z - 2.9 * x)
                   + 0.15 * torch.sin(31.0 * x + 27.0 * y + 23.0 * z))


def motion_blur(rgba: torch.Tensor, length: int) -> torch.Tensor:
    """Horizontal box blur of odd `length` pixels (borders replicated), rounded to
    uint8: the colour of a frame taken during a sideways camera motion."""
    if length <= 1:
        return rgba.clone()
    r = length // 2
    x = rgba[..., :3].to(torch.float64)
    pad = torch.cat([x[..., :1, :].expand(*x.shape[:-2], r, 3), x, x[..., -1:, :].expand(*x.shape[:-2], r, 3)], -2)
    c = torch.cumsum(torch.nn.functional.pad(pad, (0, 0, 1, 0)), dim=-2)
    box = (c[..., length:, :] - c[..., :-length, :]) / length
    out = rgba.clone()
    out[..., :3] = torch.clamp(torch.round(box), 0, 255).to(torch.uint8)
    return out


def colour_frames(scene: Scene, intr: Intrinsics, poses, config: int, *, device="cpu") -> torch.Tensor:
    """Textured colour frames [n,H,W,4] u8; about 40 % of them motion-blurred by 3-9
    pixels (seeded per config), as in hand-held RGB-D sequences."""
    _, rgba = render(scene, intr, poses, device=device, texture=True)
    g = rng(config, STREAM_BLUR)
    for k in range(rgba.shape[0]):
        if g.random() < 0.4:
            rgba[k] = motion_blur(rgba[k], int(g.choice([3, 5, 7, 9])))
    return rgba


def noise_streams(config: int):
    """The noise and invalid-mask generators of a config, for add_sensor_noise(streams=...)."""
    return rng(config, STREAM_NOISE), rng(config, STREAM_MASK)


def add_sensor_noise(depth: torch.Tensor, config: int, *, first_frame: int = 0, streams=None) -> torch.Tensor:
    """Kinect-class noise: z += N(0, sigma(z)); z outside [0.4, 4] -> 0; then 2% i.i.d.
    pixels -> 0.  Noise is drawn per frame from the config's noise / mask streams,
    frame by frame in order, so a frame's noise does not depend on batch size.
    streams: generators from noise_streams(config) that earlier calls have advanced
    to this batch's first frame (batches rendered in order); without them the streams
    are advanced to `first_frame` here (the same draws, recomputed)."""
    n, H, W = depth.shape
    if streams is not None:
        gn, gm = streams
    else:
        gn = rng(config, STREAM_NOISE)
        gm = rng(config, STREAM_MASK)
        # advance the streams to `first_frame`
        if first_frame:
            gn.standard_normal(first_frame * H * W)
            gm.random(first_frame * H * W)
    out = torch.empty_like(depth)
    for k in range(n):
        z = depth[k].double().cpu().numpy()
        eps = gn.standard_normal((H, W))
        bern = gm.random((H, W)) < INVALID_FRACTION
        zn = z + noise_sigma(z) * eps
        zn[(z <= 0) | (zn < Z_MIN) | (zn > Z_MAX) | bern] = 0.0
        out[k] = torch.from_numpy(zn.astype(np.float32)).to(depth.device)
    return out


# ----------------------------------------------------------------------------
# Scene builders
# ----------------------------------------------------------------------------

def _colour(g, shape):
    return g.integers(30, 256, size=shape, dtype=np.int64).astype(np.uint8)


def _box(cx, cy, sx, sy, z0, h):
    return np.array([cx - sx / 2, cy - sy / 2, z0, cx + sx / 2, cy + sy / 2, z0 + h])


def scene_tiny() -> Scene:
    """Room 4x4x3 m with 3 floor boxes (sides 0.3-1.0 m) and 2 spheres (r 0.2-0.4 m),
    kept clear of the 1 m camera circle about the room centre."""
    g = rng(1, STREAM_SCENE)
    boxes, spheres = [], []
    centre = np.array([2.0, 2.0])
    while len(boxes) < 3:
        sx, sy, h = g.uniform(0.3, 1.0, size=3)
        ang = g.uniform(0, 2 * math.pi)
        rad = g.uniform(1.3, 1.9)
        c = centre + rad * np.array([math.cos(ang), math.sin(ang)])
        c = np.clip(c, [sx / 2 + 0.02, sy / 2 + 0.02], [4 - sx / 2 - 0.02, 4 - sy / 2 - 0.02])
        # nearest point of the box footprint to the room centre must stay > 1.25 m away
        q = np.clip(centre, c - [sx / 2, sy / 2], c + [sx / 2, sy / 2])
        if np.linalg.norm(q - centre) > 1.25:
            boxes.append(_box(c[0], c[1], sx, sy, 0.0, h))
    while len(spheres) < 2:
        r = g.uniform(0.2, 0.4)
        ang = g.uniform(0, 2 * math.pi)
        rad = g.uniform(1.35 + r, 1.95 - 0.0)
        c = centre + rad * np.array([math.cos(ang), math.sin(ang)])
        c = np.clip(c, r + 0.02, 4 - r - 0.02)
        z = g.uniform(r, 2.0)
        if np.linalg.norm(c - centre) - r > 1.25:
            spheres.append(np.array([c[0], c[1], z, r]))
    return Scene(shell=np.array([0, 0, 0, 4, 4, 3.0]), shell_colours=_colour(g, (6, 3)),
                 boxes=np.array(boxes), box_colours=_colour(g, (3, 6, 3)),
                 spheres=np.array(spheres), sphere_colours=_colour(g, (2, 3)))


def _walls_with_doors(segments, thickness=0.1, height=3.0):
    """Interior walls as thin boxes.  segments: (axis, coord, lo, hi, [door gaps (a,b)])."""
    out = []
    for axis, coord, lo, hi, gaps in segments:
        cuts = [lo]
        for a, b in sorted(gaps):
            cuts += [a, b]
        cuts.append(hi)
        for a, b in zip(cuts[0::2], cuts[1::2]):
            if b - a < 1e-6:
                continue
            if axis == 0:   # wall at x = coord, spanning y in [a, b]
                out.append(np.array([coord - thickness / 2, a, 0.0, coord + thickness / 2, b, height]))
            else:           # wall at y = coord, spanning x in [a, b]
                out.append(np.array([a, coord - thickness / 2, 0.0, b, coord + thickness / 2, height]))
    return out


def _scatter_objects(g, n, area_lo, area_hi, keep_clear, scene_walls):
    """Random boxes and vertical cylinders (alternating) on the floor."""
    boxes, cyls = [], []
    tries = 0
    while len(boxes) + len(cyls) < n and tries < 100000:
        tries += 1
        c = g.uniform(area_lo, area_hi)
        if keep_clear(c):
            continue
        if (len(boxes) + len(cyls)) % 2 == 0:
            sx, sy = g.uniform(0.3, 1.2, size=2)
            h = g.uniform(0.3, 2.0)
            b = _box(c[0], c[1], sx, sy, 0.0, h)
            corners = [np.array([b[0], b[1]]), np.array([b[3], b[4]]),
                       np.array([b[0], b[4]]), np.array([b[3], b[1]])]
            if any(keep_clear(q) for q in corners):
                continue
            boxes.append(b)
        else:
            r = g.uniform(0.1, 0.4)
            h = g.uniform(0.5, 2.0)
            if any(keep_clear(c + r * np.array([math.cos(a), math.sin(a)])) for a in np.linspace(0, 6.28, 8)):
                continue
            cyls.append(np.array([c[0], c[1], r, 0.0, h]))
    return boxes, cyls


def scene_kinect() -> tuple[Scene, callable]:
    """10x8x3 m multi-room scene: interior walls with door gaps, 40 boxes/cylinders.
    Returns the scene and the camera path's keep-clear test."""
    g = rng(2, STREAM_SCENE)
    walls = _walls_with_doors([
        (0, 5.0, 0.0, 8.0, [(1.9, 3.1), (5.5, 6.5)]),
        (1, 4.0, 0.0, 4.95, [(2.0, 3.0)]),
        (1, 4.0, 5.05, 10.0, [(7.0, 8.0)]),
    ])

    def keep_clear(p):
        return (1.5 <= p[0] <= 8.5) and abs(p[1] - 2.5) < 0.75

    boxes, cyls = _scatter_objects(g, 40, [0.3, 0.3], [9.7, 7.7], keep_clear, walls)
    allb = np.array(walls + boxes)
    scene = Scene(shell=np.array([0, 0, 0, 10, 8, 3.0]), shell_colours=_colour(g, (6, 3)),
                  boxes=allb, box_colours=_colour(g, (len(allb), 6, 3)),
                  cylinders=np.array(cyls).reshape(-1, 5), cylinder_colours=_colour(g, (len(cyls), 2, 3)))
    return scene, keep_clear


def scene_grid(config: int = 3) -> Scene:
    """30x20x3 m grid of 6x4 rooms (5x5 m), each wall with a 1.2 m door in its middle,
    3 boxes / cylinders per room."""
    g = rng(config, STREAM_SCENE)
    segs = []
    for i in range(1, 6):
        x = 5.0 * i
        segs.append((0, x, 0.0, 20.0, [(5.0 * j + 1.9, 5.0 * j + 3.1) for j in range(4)]))
    for j in range(1, 4):
        y = 5.0 * j
        segs.append((1, y, 0.0, 30.0, [(5.0 * i + 1.9, 5.0 * i + 3.1) for i in range(6)]))
    walls = _walls_with_doors(segs)
    boxes, cyls = [], []
    for i in range(6):
        for j in range(4):
            lo = np.array([5.0 * i + 0.4, 5.0 * j + 0.4])
            hi = lo + 4.2

            def keep_clear(p, i=i, j=j):
                # keep door lanes and the room centre free
                cx, cy = 5.0 * i + 2.5, 5.0 * j + 2.5
                return abs(p[0] - cx) < 0.9 or abs(p[1] - cy) < 0.9
            b, c = _scatter_objects(g, 3, lo, hi, keep_clear, walls)
            boxes += b
            cyls += c
    allb = np.array(walls + boxes)
    return Scene(shell=np.array([0, 0, 0, 30, 20, 3.0]), shell_colours=_colour(g, (6, 3)),
                 boxes=allb, box_colours=_colour(g, (len(allb), 6, 3)),
                 cylinders=np.array(cyls).reshape(-1, 5), cylinder_colours=_colour(g, (len(cyls), 2, 3)))


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    intr: Intrinsics
    voxel_size: float
    trunc: float
    n_buckets: int
    scene: Scene
    kf_poses: np.ndarray                  # [K,3,4] poses the keyframes are integrated at
    kf_depth: torch.Tensor | None = None  # [K,H,W] f32 keyframe depth (rendered directly)
    kf_rgba: torch.Tensor | None = None   # [K,H,W,4] u8
    new_poses: np.ndarray | None = None   # [K,3,4] updated poses (pose-graph update)
    update_ids: np.ndarray | None = None  # keyframes re-integrated by the update
    frames_depth: torch.Tensor | None = None  # [N,H,W] raw frames (fusion input)
    frames_rgba: torch.Tensor | None = None
    frame_poses: np.ndarray | None = None     # [N,3,4] true frame poses
    kappa: int = 1
    updates: list = field(default_factory=list)  # batching: list of dicts(new_poses, n)
    extra: dict = field(default_factory=dict)


def workload_tiny(device="cpu") -> Workload:
    """Plain method, tiny: 4x4x3 m room, 10 keyframes of 320x240 on a 1 m-radius circle
    at 1.5 m height, looking outward with 10 deg downward pitch; voxel 2 cm, truncation
    8 cm, 2^16 buckets; 3 seeded keyframes perturbed by 1 deg / 2 cm."""
    scene = scene_tiny()
    K = 10
    poses = np.stack([look_pose(np.array([2.0 + math.cos(2 * math.pi * k / K),
                                          2.0 + math.sin(2 * math.pi * k / K), 1.5]),
                                2 * math.pi * k / K, math.radians(10.0)) for k in range(K)])
    depth, rgba = render(scene, QVGA, poses, device=device)
    depth = add_sensor_noise(depth, 1)
    gp = rng(1, STREAM_PERTURB)
    ids = np.sort(gp.choice(K, size=3, replace=False))
    new = poses.copy()
    for i in ids:
        new[i] = perturb_pose(poses[i], math.radians(1.0), 0.02, gp)
    return Workload("tiny", QVGA, 0.02, 0.08, 1 << 16, scene, poses.astype(np.float32),
                    depth, rgba, new.astype(np.float32), ids)


def kinect_trajectory(n_frames=600) -> np.ndarray:
    """Smooth path from (2.3, 2.5) to (7.7, 2.5) through a door, <= 1 cm and <= 0.5 deg
    per frame."""
    out = []
    for k in range(n_frames):
        s = k / (n_frames - 1)
        ph = 2 * math.pi * k / n_frames
        pos = np.array([2.3 + 5.4 * s, 2.5 + 0.25 * math.sin(ph), 1.5 + 0.1 * math.sin(2 * ph)])
        yaw = 0.7 * math.sin(ph + 0.3)
        pitch = math.radians(15.0) + math.radians(5.0) * math.sin(ph)
        out.append(look_pose(pos, yaw, pitch))
    return np.stack(out)


def drift_poses(poses, angle, shift, g) -> np.ndarray:
    """Random-walk drift: keyframe k is moved by the composition of k+1 random steps of
    `angle` rad / `shift` m (left-multiplied, about the camera centre)."""
    out = []
    Racc = np.eye(3)
    tacc = np.zeros(3)
    for T in poses:
        step = perturb_pose(np.hstack([np.eye(3), np.zeros((3, 1))]), angle, shift, g)
        Racc = step[:, :3] @ Racc
        tacc = tacc + step[:, 3]
        D = np.array(T, np.float64).copy()
        D[:, :3] = Racc @ D[:, :3]
        D[:, 3] = D[:, 3] + tacc
        out.append(D)
    return np.stack(out)


def workload_kinect(device="cpu", n_frames=600, kappa=10, render_frames=None, textured=False) -> Workload:
    """Plain method at Kinect scale: 600 raw 640x480 frames fused 10 per keyframe into 60
    keyframes (keyframe pose = first frame of its group), integrated at drifted poses
    (0.2 deg / 0.5 cm random walk per keyframe); one pose update moves all 60 to their
    true poses.  Voxel 1 cm, truncation 4 cm, 2^20 buckets.  render_frames renders only
    that many leading frames (the poses of all frames and keyframes are still made).
    textured=True gives the frames the colour of colour_frames (texture, seeded motion
    blur)."""
    scene, _ = scene_kinect()
    frame_poses = kinect_trajectory(n_frames)
    nr = n_frames if render_frames is None else render_frames
    fd, fr = render(scene, KINECT, frame_poses[:nr], device=device, texture=textured)
    if textured:
        g = rng(2, STREAM_BLUR)
        for k in range(fr.shape[0]):
            if g.random() < 0.4:
                fr[k] = motion_blur(fr[k], int(g.choice([3, 5, 7, 9])))
    fd = add_sensor_noise(fd, 2)
    kf_true = frame_poses[::kappa]
    g = rng(2, STREAM_PERTURB)
    kf_drift = drift_poses(kf_true, math.radians(0.2), 0.005, g)
    K = len(kf_true)
    return Workload("kinect", KINECT, 0.01, 0.04, 1 << 20, scene,
                    kf_drift.astype(np.float32), None, fr[::kappa].contiguous(),
                    kf_true.astype(np.float32), np.arange(K),
                    frames_depth=fd, frames_rgba=fr, frame_poses=frame_poses.astype(np.float32),
                    kappa=kappa)


def grid_keyframe_poses(scene: Scene, n: int, g: np.random.Generator) -> np.ndarray:
    """Seeded keyframe poses spread over the room grid: random room, free position,
    random heading, pitch in [-10, 30] deg down, height 1.0-2.0 m."""
    out = []
    while len(out) < n:
        i, j = g.integers(0, 6), g.integers(0, 4)
        p = np.array([5.0 * i + g.uniform(0.6, 4.4), 5.0 * j + g.uniform(0.6, 4.4), g.uniform(1.0, 2.0)])
        if scene.inside_solid(p, margin=0.45):
            continue
        out.append(look_pose(p, g.uniform(0, 2 * math.pi), math.radians(g.uniform(-10.0, 30.0))))
    return np.stack(out)


def workload_batching(device="cpu", n_keyframes=2000, n_updates=10, intr: Intrinsics = KINECT,
                      render_batch=64) -> Workload:
    """Batching: 2000 keyframes over a 30x20x3 m room grid, rendered directly at their
    true poses; integrated at drifted poses; 10 pose-graph updates, each re-integrating
    a seeded n in [10, 200] keyframes.  Update u moves every keyframe towards its true
    pose (drift shrinks by a seeded factor, plus a loop-closure-style jump) so that the
    largest-pose-change selection picks a spread of keyframes."""
    scene = scene_grid(3)
    gt = rng(3, STREAM_TRAJ)
    poses = grid_keyframe_poses(scene, n_keyframes, gt)
    depth = torch.empty((n_keyframes, intr.height, intr.width), dtype=torch.float32, device=device)
    rgba = torch.empty((n_keyframes, intr.height, intr.width, 4), dtype=torch.uint8, device=device)
    streams = noise_streams(3)  # batches in order: each continues the previous one's draws
    for s in range(0, n_keyframes, render_batch):
        # primitives beyond 6 m cannot give a valid (<= 4 m) depth (see render)
        d, c = render(scene, intr, poses[s:s + render_batch], device=device,
                      dtype=torch.float32 if str(device).startswith("cuda") else torch.float64, cull_radius=6.0)
        depth[s:s + render_batch] = add_sensor_noise(d, 3, streams=streams)
        rgba[s:s + render_batch] = c
    gp = rng(3, STREAM_PERTURB)
    drifted = drift_poses(poses, math.radians(0.05), 0.002, gp)
    updates = []
    cur = drifted.copy()
    for u in range(n_updates):
        n = int(gp.integers(10, 201))
        frac = gp.uniform(0.3, 0.8)
        tgt = []
        for k in range(n_keyframes):
            T = np.array(cur[k]).copy()
            # blend translation towards the truth and re-perturb slightly
            T[:, 3] = poses[k][:, 3] + frac * (cur[k][:, 3] - poses[k][:, 3])
            T = perturb_pose(T, math.radians(gp.uniform(0, 0.3)), gp.uniform(0, 0.01), gp)
            tgt.append(T)
        updates.append({"target_poses": np.stack(tgt).astype(np.float32), "n": n})
        cur = np.stack(tgt)
    return Workload("batching", intr, 0.01, 0.04, 1 << 22, scene, drifted.astype(np.float32),
                    depth, rgba, poses.astype(np.float32), None, updates=updates)


def surface_points(scene: Scene, n: int, config: int, lo=None, hi=None) -> np.ndarray:
    """n points sampled uniformly by area on the scene's analytic surfaces (shell walls,
    floor, ceiling, box faces, spheres, cylinder sides and tops), optionally restricted to
    an axis-aligned region [lo, hi].  Returns float64 [n, 3]."""
    g = rng(config, STREAM_POINTS)
    pieces = []   # (area, sampler)

    def rect(axis, coord, a0, a1, b0, b1):
        area = (a1 - a0) * (b1 - b0)

        def smp(m):
            a = g.uniform(a0, a1, m)
            b = g.uniform(b0, b1, m)
            c = np.full(m, coord)
            if axis == 0:
                return np.stack([c, a, b], 1)
            if axis == 1:
                return np.stack([a, c, b], 1)
            return np.stack([a, b, c], 1)
        return area, smp

    def box_faces(b, skip_bottom=True):
        x0, y0, z0, x1, y1, z1 = b
        out = [rect(0, x0, y0, y1, z0, z1), rect(0, x1, y0, y1, z0, z1),
               rect(1, y0, x0, x1, z0, z1), rect(1, y1, x0, x1, z0, z1),
               rect(2, z1, x0, x1, y0, y1)]
        if not skip_bottom:
            out.append(rect(2, z0, x0, x1, y0, y1))
        return out

    pieces += box_faces(scene.shell, skip_bottom=False)
    for b in scene.boxes:
        pieces += box_faces(b)
    for s in scene.spheres:
        def smp(m, s=s):
            v = g.normal(size=(m, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            return s[:3] + s[3] * v
        pieces.append((4 * math.pi * s[3] ** 2, smp))
    for c in scene.cylinders:
        def smp_side(m, c=c):
            a = g.uniform(0, 2 * math.pi, m)
            z = g.uniform(c[3], c[4], m)
            return np.stack([c[0] + c[2] * np.cos(a), c[1] + c[2] * np.sin(a), z], 1)

        def smp_top(m, c=c):
            r = c[2] * np.sqrt(g.uniform(0, 1, m))
            a = g.uniform(0, 2 * math.pi, m)
            return np.stack([c[0] + r * np.cos(a), c[1] + r * np.sin(a), np.full(m, c[4])], 1)
        pieces.append((2 * math.pi * c[2] * (c[4] - c[3]), smp_side))
        pieces.append((math.pi * c[2] ** 2, smp_top))
    areas = np.array([a for a, _ in pieces])
    counts = g.multinomial(n * 4 if lo is not None else n, areas / areas.sum())
    pts = np.concatenate([smp(m) for (_, smp), m in zip(pieces, counts) if m > 0], 0)
    if lo is not None:
        keep = np.all((pts >= lo) & (pts <= hi), axis=1)
        pts = pts[keep]
    g.shuffle(pts)
    return pts[:n]
