"""The fusion weight's normal (Eq. 1, w_z = cos(theta) / Z^2) in the expanded form the
fusion kernel evaluates, checked against its definition: the cross product of the two
central differences of back-projected points.  Pure numpy, no GPU.

With r = (xn, yn, 1), A = (z_r + z_l) / fx and B = (z_d + z_u) / fy,
    a = P(u+1, v) - P(u-1, v) = (z_r - z_l) r + (A, 0, 0)
    b = P(u, v+1) - P(u, v-1) = (z_d - z_u) r + (0, B, 0)
and a x b = (-(z_r - z_l) B, -(z_d - z_u) A, A B + (z_r - z_l) B xn + (z_d - z_u) A yn)."""
import numpy as np


def _backproject(u, v, z, fx, fy, cx, cy):
    return np.stack([(u - cx) / fx * z, (v - cy) / fy * z, z], axis=-1)


def _cases(n, seed):
    g = np.random.default_rng(seed)
    fx, fy, cx, cy = 525.0, 525.0, 319.5, 239.5
    u = g.integers(1, 639, n).astype(np.float64)
    v = g.integers(1, 479, n).astype(np.float64)
    z = g.uniform(0.4, 6.0, n)
    # depth steps from fronto-parallel to grazing: up to 30x the pixel footprint z / f
    sx = g.uniform(-30, 30, n) * z / fx
    sy = g.uniform(-30, 30, n) * z / fy
    e = g.normal(0, 1e-3, (4, n)) * z / fx      # sensor-like noise on each neighbour
    zl, zr = z - sx + e[0], z + sx + e[1]
    zu, zd = z - sy + e[2], z + sy + e[3]
    return (fx, fy, cx, cy), u, v, z, zl, zr, zu, zd


def _cos_definition(K, u, v, zl, zr, zu, zd):
    fx, fy, cx, cy = K
    a = _backproject(u + 1, v, zr, *K) - _backproject(u - 1, v, zl, *K)
    b = _backproject(u, v + 1, zd, *K) - _backproject(u, v - 1, zu, *K)
    n = np.cross(a, b)
    return np.abs(n[:, 2]) / np.linalg.norm(n, axis=1)


def _cos_expanded(K, u, v, zl, zr, zu, zd, dtype):
    fx, fy, cx, cy = (dtype(k) for k in K)
    t = lambda x: np.asarray(x, dtype)
    u, v, zl, zr, zu, zd = map(t, (u, v, zl, zr, zu, zd))
    one = dtype(1)
    xn = (u - cx) * (one / fx)
    yn = (v - cy) * (one / fy)
    A = (zr + zl) * (one / fx)
    B = (zd + zu) * (one / fy)
    m1 = (zr - zl) * B
    m2 = (zd - zu) * A
    nz = m1 * xn + (m2 * yn + A * B)
    n2 = m1 * m1 + (m2 * m2 + nz * nz)
    return np.abs(nz) / np.sqrt(n2)


def test_expansion_equals_the_cross_product_in_double():
    K, u, v, z, zl, zr, zu, zd = _cases(20000, 3)
    ref = _cos_definition(K, u, v, zl, zr, zu, zd)
    got = _cos_expanded(K, u, v, zl, zr, zu, zd, np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-12


def _cos_cross_float32(K, u, v, zl, zr, zu, zd):
    """The cross product of the two differences formed in float32 (no expansion)."""
    f = np.float32
    fx, fy, cx, cy = (f(k) for k in K)
    zl, zr, zu, zd = (np.asarray(x, f) for x in (zl, zr, zu, zd))
    xn = (u.astype(f) - cx) * (f(1) / fx)
    yn = (v.astype(f) - cy) * (f(1) / fy)
    dzx, dzy = zr - zl, zd - zu
    a = (xn * dzx + (zr + zl) * (f(1) / fx), yn * dzx, dzx)
    b = (xn * dzy, yn * dzy + (zd + zu) * (f(1) / fy), dzy)
    n = (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])
    return np.abs(n[2]) / np.sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2])


def test_expansion_in_float32_keeps_cos_theta_at_grazing_angles():
    # the float32 evaluation never forms the cancelling (z_r - z_l)(z_d - z_u) xn yn
    # terms of a_x b_y and a_y b_x, so its cos(theta) error stays near 1e-7 absolute at
    # every angle, about ten times below the cross product formed in float32
    K, u, v, z, zl, zr, zu, zd = _cases(20000, 4)
    zs = [np.float32(x).astype(np.float64) for x in (zl, zr, zu, zd)]   # float32 depth inputs
    ref = _cos_definition(K, u, v, *zs)
    got = _cos_expanded(K, u, v, *zs, np.float32).astype(np.float64)
    naive = _cos_cross_float32(K, u, v, *zs).astype(np.float64)
    assert ref.min() < 1e-3                        # the cases reach grazing angles
    err = np.abs(got - ref)
    assert err.max() <= 2e-7
    # relative to cos(theta) itself, wherever the surface is not seen edge-on (there the
    # three terms of n_z cancel by geometry, not by rounding)
    assert (err / ref)[ref >= 1e-2].max() <= 1e-5
    assert np.abs(naive - ref).max() > 4 * err.max()


def test_fronto_parallel_plane_has_cos_theta_one():
    K = (525.0, 525.0, 319.5, 239.5)
    u = np.array([1.0, 319.0, 638.0])
    v = np.array([1.0, 239.0, 478.0])
    z = np.full(3, 2.0)
    # a plane at constant depth: the normal is the optical axis wherever the pixel is
    got = _cos_expanded(K, u, v, z, z, z, z, np.float64)
    assert np.allclose(got, 1.0, atol=1e-15)
