"""Small closed-form scenes for the oracle pins (input construction only)."""
import numpy as np


def identity_pose():
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = np.eye(3)
    return T


def plane_depth(intr, z0):
    fx, fy, cx, cy, W, H = intr
    return np.full((H, W), np.float32(z0), np.float32)


def uniform_rgba(intr, rgb):
    fx, fy, cx, cy, W, H = intr
    a = np.zeros((H, W, 4), np.uint8)
    a[..., :3] = rgb
    a[..., 3] = 255
    return a


def sphere_depth(intr, centre, radius):
    """z-depth of the first ray-sphere hit at each pixel centre (closed form), 0 = miss."""
    fx, fy, cx, cy, W, H = intr
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    d = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1)
    return sphere_hit_z(d, centre, radius).astype(np.float32)


def sphere_hit_z(d, centre, radius):
    c = np.asarray(centre, float)
    a = (d * d).sum(-1)
    b = -2.0 * (d * c).sum(-1)
    cc = (c * c).sum() - radius ** 2
    disc = b * b - 4 * a * cc
    lam = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
    return np.where(disc >= 0, lam, 0.0)


def voxel_positions(coords, s):
    """World positions [n,512,3] of every voxel of blocks `coords` [n,3] (voxel i at i*s,
    linear index x + 8y + 64z inside a block)."""
    l = np.arange(512)
    lx, ly, lz = l % 8, (l // 8) % 8, l // 64
    base = coords[:, None, :].astype(np.int64) * 8
    idx = base + np.stack([lx, ly, lz], -1)[None]
    return idx * s
