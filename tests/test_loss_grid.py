"""The loss's grid coordinate g = p / s (the voxel cell of a point and its fraction,
which set the trilinear weights) as the point pass evaluates it in float32 -- a quotient
q = p (1/s), its residual r = p - q s from one fused multiply-add, fraction
(q - floor(q)) + r / s -- against the exact quotient in double.  Pure numpy, no GPU;
the fused multiply-add is evaluated exactly in double and rounded once to float32."""
import numpy as np

f32 = np.float32


def _kernel_grid(x, s):
    """floor and fraction of x / s in the point pass's float32 steps."""
    inv_s = f32(1.0 / np.float64(s))
    q = (x * inv_s).astype(f32)
    r = (x.astype(np.float64) - q.astype(np.float64) * np.float64(s)).astype(f32)  # fma(-q, s, x)
    fl = np.floor(q)
    fr = ((q - fl).astype(f32) + (r * inv_s).astype(f32)).astype(f32)
    lo = fr < 0
    fl[lo] -= f32(1)
    fr[lo] += f32(1)
    hi = fr >= 1
    fl[hi] += f32(1)
    fr[hi] -= f32(1)
    return fl.astype(np.int64), fr.astype(np.float64)


def _exact_grid(x, s):
    g = x.astype(np.float64) / np.float64(s)
    fl = np.floor(g)
    return fl.astype(np.int64), g - fl


def _points(n, seed, half_extent):
    g = np.random.default_rng(seed)
    return g.uniform(-half_extent, half_extent, n).astype(f32)


def test_cell_and_fraction_match_the_exact_quotient():
    s = f32(0.01)
    for extent in (1.0, 20.0, 80.0):          # up to 8000 voxels from the origin
        x = _points(200000, int(extent), extent)
        fl, fr = _kernel_grid(x, s)
        fle, fre = _exact_grid(x, s)
        # away from a cell face (where the oracle flags a point as marginal) the cell is
        # the same and the fraction is within about half a float32 ulp of 1 (6e-8 voxel)
        clear = np.minimum(fre, 1 - fre) > 1e-6
        assert clear.mean() > 0.99
        assert np.array_equal(fl[clear], fle[clear])
        assert np.abs(fr - fre)[clear].max() <= 1e-7
        # at a face either neighbouring cell interpolates the same value: the position
        # fl + fr agrees with g everywhere
        assert np.abs((fl + fr) - (fle + fre)).max() <= 1e-7


def test_a_float32_quotient_alone_is_not_enough_far_from_the_origin():
    # the reason for the residual: at thousands of voxels from the origin a float32
    # grid coordinate carries about 1e-4 voxel of error in the fraction
    s = f32(0.01)
    x = _points(200000, 9, 80.0)
    q = (x * f32(1.0 / np.float64(s))).astype(f32).astype(np.float64)
    fle, fre = _exact_grid(x, s)
    assert np.abs((q - np.floor(q)) - fre)[np.minimum(fre, 1 - fre) > 1e-3].max() > 1e-4


def test_points_on_and_halfway_between_grid_points():
    s = f32(0.01)
    k = np.arange(-5000, 5000, 37, dtype=np.int64)
    on = (k.astype(f32) * s).astype(f32)            # float32 products: near, not exactly, k s
    fl, fr = _kernel_grid(on, s)
    fle, fre = _exact_grid(on, s)
    assert np.abs((fl + fr) - (fle + fre)).max() <= 1e-7
    mid = ((k.astype(np.float64) + 0.5) * np.float64(s)).astype(f32)
    fl, fr = _kernel_grid(mid, s)
    assert np.array_equal(fl, k) and np.abs(fr - 0.5).max() < 1e-3
