"""Pins of the oracle's forward light-tracing splat (Sec. 3, Eq. 8): hand
cases of the tent pixel filter, the per-pixel brute-force formulation,
conservation of the deposited weight and the multiplicative role of I and
G = d_z."""
import numpy as np

from oracle import splat as S

W, H, PX = 8, 6, 0.5


def centre(i, j):
    return (i + 0.5 - W / 2) * PX, (j + 0.5 - H / 2) * PX


def one(x, y, dz=1.0, I=1.0, weight=1.0):
    return S.splat([x], [y], [dz], [I], [1], W, H, PX, weight)


def test_ray_at_a_pixel_centre_deposits_everything_there():
    x, y = centre(3, 2)
    img = one(x, y, dz=0.8, I=0.5, weight=2.0)
    assert img[2, 3] == 0.8 * 0.5 * 2.0
    assert np.count_nonzero(img) == 1


def test_ray_at_a_pixel_corner_splits_in_four():
    x0, y0 = centre(3, 2)
    img = one(x0 + PX / 2, y0 + PX / 2)
    np.testing.assert_allclose(img[2:4, 3:5], 0.25, rtol=0, atol=1e-15)
    assert abs(img.sum() - 1.0) < 1e-15


def test_quarter_pixel_offset_splits_three_to_one():
    x0, y0 = centre(4, 1)
    img = one(x0 + PX / 4, y0)
    assert abs(img[1, 4] - 0.75) < 1e-15 and abs(img[1, 5] - 0.25) < 1e-15


def test_matches_brute_force_tent_filter():
    rng = np.random.default_rng(7)
    n = 300
    x = rng.uniform(-W * PX / 2 - PX, W * PX / 2 + PX, n)     # some fall off the sensor
    y = rng.uniform(-H * PX / 2 - PX, H * PX / 2 + PX, n)
    dz = rng.uniform(0.2, 1.0, n)
    I = rng.uniform(0.0, 1.0, n)
    valid = rng.uniform(size=n) < 0.8
    a = S.splat(x, y, dz, I, valid, W, H, PX, 0.3)
    b = S.splat_brute(x, y, dz, I, valid, W, H, PX, 0.3)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_weight_is_conserved_inside_the_sensor():
    rng = np.random.default_rng(8)
    n = 500
    x = rng.uniform(-(W / 2 - 1) * PX, (W / 2 - 1) * PX, n)
    y = rng.uniform(-(H / 2 - 1) * PX, (H / 2 - 1) * PX, n)
    dz = rng.uniform(0.2, 1.0, n)
    I = rng.uniform(0.0, 1.0, n)
    img = S.splat(x, y, dz, I, np.ones(n), W, H, PX, 1.0 / n)
    assert abs(img.sum() - (I * dz).sum() / n) < 1e-13


def test_throughput_and_geometric_factor_multiply():
    x, y = centre(2, 2)
    x += 0.1 * PX
    base = one(x, y, dz=0.5, I=0.25)
    np.testing.assert_allclose(one(x, y, dz=1.0, I=0.25), 2 * base, rtol=1e-15)
    np.testing.assert_allclose(one(x, y, dz=0.5, I=0.75), 3 * base, rtol=1e-15)


def test_invalid_rays_deposit_nothing():
    x, y = centre(1, 1)
    img = S.splat([x], [y], [1.0], [1.0], [0], W, H, PX)
    assert not img.any()


def test_mirror_symmetry():
    rng = np.random.default_rng(9)
    n = 50
    x = rng.uniform(-W * PX / 2, W * PX / 2, n)
    y = rng.uniform(-H * PX / 2, H * PX / 2, n)
    a = S.splat(x, y, np.ones(n), np.ones(n), np.ones(n), W, H, PX)
    b = S.splat(-x, y, np.ones(n), np.ones(n), np.ones(n), W, H, PX)
    np.testing.assert_allclose(a[:, ::-1], b, rtol=0, atol=1e-13)


def test_deposit_bound_covers_shifted_hits():
    """Moving every hit by up to pos_tol and every I, d_z by up to val_tol
    keeps each pixel within the bound."""
    rng = np.random.default_rng(10)
    n = 400
    x = rng.uniform(-W * PX / 2, W * PX / 2, n)
    y = rng.uniform(-H * PX / 2, H * PX / 2, n)
    dz = rng.uniform(0.2, 1.0, n)
    I = rng.uniform(0.0, 1.0, n)
    v = np.ones(n)
    pos_tol, val_tol = 1e-3, 1e-4
    a = S.splat(x, y, dz, I, v, W, H, PX, 0.5)
    b = S.splat(x + rng.uniform(-pos_tol, pos_tol, n), y + rng.uniform(-pos_tol, pos_tol, n),
                dz + rng.uniform(-val_tol, val_tol, n), I + rng.uniform(-val_tol, val_tol, n), v, W, H, PX, 0.5)
    bound = S.deposit_bound(x, y, dz, I, v, W, H, PX, 0.5, pos_tol, val_tol)
    assert np.all(np.abs(a - b) <= bound + 1e-15)
