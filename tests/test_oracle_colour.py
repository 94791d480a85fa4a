"""Oracle pins for colour keyframe fusion (Section 3 "Keyframe Fusion", colour paragraph):
unsharp masking, the per-frame blurriness weight w_b, the back-warp with bilinear
sampling, the colour weight w_c = w_b * w_z and the weighted median.

Every expected value below is a closed form, an invariant of the definition, or a
brute-force characterisation that shares no arithmetic with the oracle."""
import math

import numpy as np
import pytest

import oracle
from oracle_helpers import identity_pose, plane_depth

INTR = (60.0, 60.0, 31.5, 23.5, 64, 48)
H, W = 48, 64


def gray(img):
    """[H,W] gray levels -> [H,W,4] uint8 (R = G = B, alpha 255)."""
    a = np.zeros(img.shape + (4,), np.uint8)
    a[..., :3] = np.asarray(img, np.uint8)[..., None]
    a[..., 3] = 255
    return a


def edge_image(width, height=252, at=24, shape=(H, W), lo=0):
    """Vertical edge: gray lo left of column `at`, rising linearly by height/width per
    column over `width` columns, lo + height after."""
    x = np.arange(shape[1])
    prof = lo + np.clip((x - at + 1) * (height // width), 0, height)
    return np.broadcast_to(prof, shape).copy()


# ------------------------------------------------------------------ unsharp masking

def test_unsharp_leaves_constant_image():
    S = oracle.unsharp(gray(np.full((H, W), 97)))
    assert np.all(S == 97.0)


def test_unsharp_quadratic_loses_the_filter_variance():
    # the binomial (1 4 6 4 1)/16 has variance 1 per axis: G*x^2 = x^2 + 1 away from the
    # borders, so the unsharp image is 2 x^2 - (x^2 + 1) = x^2 - 1 (and likewise per axis)
    n = 12
    y, x = np.mgrid[0:n, 0:n]
    S = oracle.unsharp(gray(x * x))
    assert np.array_equal(S[:, 2:n - 2, 0], (x * x - 1.0)[:, 2:n - 2])
    S = oracle.unsharp(gray(y * y))
    assert np.array_equal(S[2:n - 2, :, 1], (y * y - 1.0)[2:n - 2, :])
    S = oracle.unsharp(gray(x * x + y * y))
    assert np.array_equal(S[2:n - 2, 2:n - 2, 2], (x * x + y * y - 2.0)[2:n - 2, 2:n - 2])


def test_unsharp_leaves_linear_interior_and_clamps():
    y, x = np.mgrid[0:H, 0:W]
    img = x + 2 * y
    S = oracle.unsharp(gray(img))
    assert np.array_equal(S[2:-2, 2:-2, 0], img[2:-2, 2:-2].astype(float))
    dot = np.zeros((H, W), int)
    dot[20, 30] = 255
    S = oracle.unsharp(gray(dot))
    assert S.min() == 0.0 and S.max() == 255.0 and S[20, 30, 0] == 255.0
    # the ring around the dot would go negative without the clamp
    assert S[20, 31, 0] == 0.0


def test_unsharp_channels_are_independent():
    rgba = np.zeros((H, W, 4), np.uint8)
    rgba[..., 0] = 40
    rgba[:, 32:, 1] = 200
    S = oracle.unsharp(rgba)
    assert np.all(S[..., 0] == 40.0) and np.all(S[..., 2] == 0.0)
    assert S[:, 31, 1].max() == 0.0 and S[:, 32, 1].min() == 255.0


# ------------------------------------------------------------------ blurriness

def _ramp_blurriness(s):
    """Closed form for an edge rising by h/s per column over s columns: D_F = h/s on the
    ramp columns, and the box mean's difference at column j is (1/9) of the ramp
    differences inside the window [j-4, j+4].  So V_j = (h/s)(1 - n_j/9) with n_j the
    ramp columns in that window, and b = sum_j n_j / (9 s)."""
    n = [min(j + 4, s - 1) - max(j - 4, 0) + 1 for j in range(s)]
    return sum(n) / (9.0 * s)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 6, 7, 9])
def test_blurriness_of_ramp_edge(s):
    # up to width 5 every window holds the whole ramp: b = s / 9; wider ramps keep less
    img = edge_image(s)
    expect = s / 9.0 if s <= 5 else _ramp_blurriness(s)
    assert abs(_ramp_blurriness(s) - expect) < 1e-15
    assert abs(oracle.blurriness(gray(img)) - expect) < 1e-12
    assert abs(oracle.blurriness(gray(img.T.copy())) - expect) < 1e-12


def test_blurriness_takes_the_blurrier_direction():
    # f(x, y) = g1(x) + g2(y): each direction sees only its own edge
    gx = edge_image(2, height=124)
    gy = edge_image(4, height=124, at=20, shape=(W, H)).T
    assert abs(oracle.blurriness(gray(gx + gy)) - 4.0 / 9.0) < 1e-12
    gy2 = edge_image(1, height=124, at=20, shape=(W, H)).T
    assert abs(oracle.blurriness(gray(gx + gy2)) - 2.0 / 9.0) < 1e-12


def test_blurriness_uses_the_luma_weights():
    # R rising by 150 while G falls by 77 leaves Y = (77 R + 150 G + 29 B)/256 constant:
    # no luma edge, b = 0; each edge alone is an ordinary width-3 edge
    rgba = np.zeros((H, W, 4), np.uint8)
    rgba[..., 3] = 255
    # exact opposing steps (width 1) so that 77 dR = -150 dG column by column
    r = edge_image(1, height=150)
    g = 77 - edge_image(1, height=77)
    rgba[..., 0], rgba[..., 1] = r, g
    assert oracle.blurriness(rgba) == 0.0
    rgba[..., 1] = 0
    assert abs(oracle.blurriness(rgba) - 1.0 / 9.0) < 1e-12


def test_blurriness_of_flat_image_is_zero():
    assert oracle.blurriness(gray(np.full((H, W), 13))) == 0.0


# ------------------------------------------------------------------ weighted median

def _l1(values, weights, m):
    return float(np.sum(np.asarray(weights) * np.abs(np.asarray(values) - m)))


def test_weighted_median_is_the_smallest_l1_minimiser():
    # the lower weighted median minimises sum_j w_j |c_j - m|; among the sample values
    # it is the smallest minimiser
    g = np.random.default_rng(7)
    for trial in range(300):
        n = int(g.integers(1, 13))
        vals = g.integers(0, 8, n).astype(float) * 31.0 + (g.random(n) < 0.5) * g.random(n)
        w = g.random(n) + 0.01
        m = oracle.weighted_median(vals, w)
        assert m in vals
        f = [_l1(vals, w, v) for v in vals]
        fm = _l1(vals, w, m)
        assert fm <= min(f) * (1 + 1e-12) + 1e-12
        for v, fv in zip(vals, f):
            if v < m:
                assert fv > fm


def test_weighted_median_equal_weights_is_the_median():
    g = np.random.default_rng(3)
    for n in (1, 3, 5, 9):
        v = g.random(n) * 255
        assert oracle.weighted_median(v, np.ones(n)) == np.median(v)


# ------------------------------------------------------------------ fusion pipeline

def _translated(tx):
    T = identity_pose()
    T[0, 3] = tx
    return T


def test_identity_frames_sample_the_pixel_and_weight_is_wb_over_z2():
    z0 = 2.0
    y, x = np.mgrid[0:H, 0:W]
    img = gray(x + 2 * y)   # linear: unchanged by unsharp masking away from the borders
    n = 3
    out = oracle.fuse_colour(np.stack([img] * n), np.stack([plane_depth(INTR, z0)] * n),
                             np.stack([identity_pose()] * n), plane_depth(INTR, z0), identity_pose(), INTR)
    inner = (slice(2, -2), slice(2, -2))
    assert np.all(out.nobs[inner] == n)
    # the round trip pi(pi^-1(x)) is exact up to double rounding
    assert np.abs(out.median[inner][..., 0] - (x + 2 * y)[inner]).max() < 1e-9
    assert np.array_equal(out.rgba[inner][..., 1], (x + 2 * y)[inner].astype(np.uint8))
    assert np.all(out.rgba[inner][..., 3] == 255)
    # fronto-parallel plane: cos(theta) = 1, w_c = w_b / Z^2 per frame
    assert np.abs(out.wsum[inner] - out.wb.sum() / z0 ** 2).max() < 1e-12
    # the border ring has no central-difference normal: no colour
    assert np.all(out.nobs[0] == 0) and np.all(out.rgba[:, 0] == 0)


def test_translated_frames_sample_the_shifted_ramp():
    # plane at Z; frame i translated by t_i along x sees keyframe pixel u at
    # u - fx t_i / Z; on a linear ramp a*u + b*v + c_i the bilinear sample is exact
    z0, fx = 2.0, INTR[0]
    ts = [-0.02, 0.01, 0.03]
    offs = [60, 20, 40]
    y, x = np.mgrid[0:H, 0:W]
    imgs = [gray(2 * x + y + o) for o in offs]
    out = oracle.fuse_colour(np.stack(imgs), np.stack([plane_depth(INTR, z0)] * 3),
                             np.stack([_translated(t) for t in ts]), plane_depth(INTR, z0), identity_pose(),
                             INTR)
    for (v, u) in [(10, 10), (20, 30), (30, 50), (40, 20)]:
        samples = [2 * (u - fx * float(np.float32(t)) / z0) + v + o for t, o in zip(ts, offs)]
        assert out.nobs[v, u] == 3
        # equal images up to an offset -> equal w_b; equal depth and normal -> equal w_z
        assert abs(out.median[v, u, 0] - np.median(samples)) < 1e-9


def test_weights_follow_frame_blurriness():
    # constant colour c_i per frame plus an edge of width s_i <= 5 far right:
    # w_b = 1 - s_i/9, so away from the edge the colour is the weighted median of c_i
    z0 = 1.5
    cs = [30, 90, 150, 190]
    widths = [5, 1, 3, 4]
    imgs = [gray(edge_image(s, height=60, at=50) + c) for c, s in zip(cs, widths)]
    n = len(cs)
    out = oracle.fuse_colour(np.stack(imgs), np.stack([plane_depth(INTR, z0)] * n),
                             np.stack([identity_pose()] * n), plane_depth(INTR, z0), identity_pose(), INTR)
    wb = np.array([1 - s / 9.0 for s in widths])
    assert np.abs(out.wb - wb).max() < 1e-12
    fs = [_l1(cs, wb, c) for c in cs]
    expect = min(c for c, f in zip(cs, fs) if f <= min(fs) * (1 + 1e-12))
    assert expect == 90  # the sharpest frame carries the median here
    region = out.median[3:-3, 3:40, 0]
    assert np.all(region == expect)
    assert np.all(out.nobs[3:-3, 3:40] == n)


def test_tilted_plane_weight_is_cos_theta_over_z2():
    fx, fy, cx, cy, Wd, Hd = INTR
    tilt = math.radians(30.0)
    nrm = np.array([0.0, math.sin(tilt), -math.cos(tilt)])
    d0 = 1.3
    v, u = np.mgrid[0:Hd, 0:Wd].astype(np.float64)
    ray = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1)
    depth = (-d0 / (ray @ nrm)).astype(np.float32)
    img = gray(np.full((Hd, Wd), 120))   # flat: w_b = 1
    out = oracle.fuse_colour(np.stack([img] * 2), np.stack([depth] * 2), np.stack([identity_pose()] * 2),
                             depth, identity_pose(), INTR)
    inner = (slice(1, -1), slice(1, -1))
    z = depth.astype(np.float64)[inner]
    assert np.all(out.wb == 1.0)
    assert np.abs(out.wsum[inner] - 2 * math.cos(tilt) / z ** 2).max() < 1e-5 * out.wsum[inner].max()
    assert np.all(out.rgba[inner][..., 0] == 120)


def test_occluded_and_out_of_view_samples_are_dropped():
    z0, fx = 2.0, INTR[0]
    n = 3
    imgs = [gray(np.full((H, W), c)) for c in (50, 100, 200)]
    depths = [plane_depth(INTR, z0) for _ in range(n)]
    depths[2][10:20, 10:20] = 1.0   # an occluder in front of the plane in frame 2
    ts = [0.0, 0.0, 0.2]            # frame 2 shifted by fx * 0.2 / 2 = 6 px
    out = oracle.fuse_colour(np.stack(imgs), np.stack(depths), np.stack([_translated(t) for t in ts]),
                             plane_depth(INTR, z0), identity_pose(), INTR)
    shift = fx * float(np.float32(0.2)) / z0
    for v in range(2, H - 2):
        for u in range(2, W - 2):
            us = u - shift
            in_view = 0 <= us <= W - 1
            hidden = 10 <= math.floor(us + 0.5) < 20 and 10 <= v < 20
            expect = 2 + (1 if in_view and not hidden else 0)
            assert out.nobs[v, u] == expect, (v, u)
            # equal weights: two observations -> the lower one (50); three -> 100
            assert out.rgba[v, u, 0] == (100 if expect == 3 else 50)
