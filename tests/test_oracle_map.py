"""Pins for the oracle's tabulated map (paper Sec. 4.2 factorised mask +
regressor; the table is this library's regressor).  Checked against exact
properties of multilinear interpolation, the exact tracer it falls back to,
and lens geometry that fixes a cell's class by inspection."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04017_gb300 import workloads as w

SMAX = math.tan(math.radians(10.0))


def singlet():
    return oracle.Lens(w.singlet_lens())


def box(rho=12.0, smax=SMAX, lam=(380.0, 780.0)):
    return [-rho, -rho, -smax, -smax, lam[0]], [rho, rho, smax, smax, lam[1]]


def node_coords(lat, d, i):
    return np.float32(lat.lo_f[d] + np.float32(np.float32(i) * lat.step_f[d]))


def test_lattice_constants_fp32():
    lo, hi = box()
    lat = oracle.Lattice([32, 32, 32, 32, 8], lo, hi)
    assert lat.lo_f[0] == np.float32(-12.0)
    assert lat.step_f[0] == np.float32(24.0 / 31.0)
    assert lat.inv_f[4] == np.float32(7.0 / 400.0)
    assert lat.n_nodes == 32 ** 4 * 8 and lat.n_cells == 31 ** 4 * 7


def test_affine_field_is_reproduced_exactly():
    """Multilinear interpolation is exact for any affine function of the five
    coordinates; direction channels carry a constant unit vector."""
    lo, hi = box()
    lat = oracle.Lattice([7, 5, 6, 4, 3], lo, hi)
    rng = np.random.default_rng(11)
    A = rng.normal(size=(3, 5))
    b = rng.normal(size=3)
    dconst = np.array([0.2, -0.1, math.sqrt(1 - 0.05)])
    rays = w.entrance_rays(500, 5, 11.0)
    for r in range(len(rays)):
        ray = np.array([a[r] for a in rays.arrays()], np.float32)
        cell = lat.cell_of(ray)
        assert cell is not None
        corner6 = np.zeros((32, 6))
        for k in range(32):
            q = np.array([node_coords(lat, d, cell[d] + ((k >> (4 - d)) & 1)) for d in range(5)],
                         np.float64)
            f = A @ q + b
            corner6[k] = [f[0], f[1], *dconst, f[2]]
        out, c2 = lat.interpolate(corner6, ray)
        v = np.array([ray[0], ray[1], ray[2] / np.float64(ray[4]), ray[3] / np.float64(ray[4]),
                      ray[5]], np.float64)
        f = A @ v + b
        assert np.allclose(out[[0, 1, 5]], f, rtol=1e-12, atol=1e-11)
        assert np.allclose(out[2:5], dconst, atol=1e-15)


def test_multilinear_field_is_reproduced_exactly():
    """The interpolant is the tensor-product (multilinear) one, not just any
    affine-exact scheme: a product of affine factors, one per coordinate
    (x y s_x s_y lambda terms included), is reproduced exactly, which a
    simplex or other piecewise-linear interpolant would not do."""
    lo, hi = box()
    lat = oracle.Lattice([6, 7, 5, 6, 4], lo, hi)
    rng = np.random.default_rng(17)
    a = rng.normal(size=5)
    c = rng.normal(size=5) * 3.0
    scale = np.array([1 / 12.0, 1 / 12.0, 1 / SMAX, 1 / SMAX, 1 / 400.0])

    def field(q):
        return float(np.prod(c + a * q * scale))

    rays = w.entrance_rays(300, 8, 11.0)
    worst = 0.0
    for r in range(len(rays)):
        ray = np.array([x[r] for x in rays.arrays()], np.float32)
        cell = lat.cell_of(ray)
        assert cell is not None
        corner6 = np.zeros((32, 6))
        for k in range(32):
            q = np.array([node_coords(lat, d, cell[d] + ((k >> (4 - d)) & 1)) for d in range(5)],
                         np.float64)
            corner6[k] = [field(q), 0.0, 0.0, 0.0, 1.0, 0.0]
        out, _ = lat.interpolate(corner6, ray)
        v = np.array([ray[0], ray[1], ray[2] / np.float64(ray[4]), ray[3] / np.float64(ray[4]),
                      ray[5]], np.float64)
        want = field(v)
        worst = max(worst, abs(out[0] - want) / (1 + abs(want)))
    assert worst < 1e-11


def test_query_at_a_node_returns_the_node_value():
    lo, hi = box()
    lat = oracle.Lattice([5, 5, 5, 5, 3], lo, hi)
    rng = np.random.default_rng(2)
    for _ in range(50):
        idx = rng.integers(0, [4, 4, 4, 4, 2])
        ray = lat.node_ray(idx)
        cell = lat.cell_of(ray)
        assert cell is not None
        corner6 = rng.normal(size=(32, 6))
        corner6[:, 2:5] = [0, 0, 1]
        out, _ = lat.interpolate(corner6, ray)
        k = sum(((idx[d] - cell[d]) & 1) << (4 - d) for d in range(5))
        assert np.allclose(out[[0, 1, 5]], corner6[k, [0, 1, 5]], rtol=1e-6, atol=1e-6)


def test_cell_index_is_fp32_rule():
    """The cell of a ray uses FP32 slopes and FP32 (v - lo) * inv_step."""
    lo, hi = box()
    lat = oracle.Lattice([32, 32, 32, 32, 8], lo, hi)
    rays = w.singlet_rays(2000)
    ids = lat.cell_ids(rays)
    f = np.float32
    for r in range(0, 2000, 7):
        v = [rays.x[r], rays.y[r], f(rays.dx[r] / rays.dz[r]), f(rays.dy[r] / rays.dz[r]),
             rays.lam[r]]
        u = [f(f(v[d] - lat.lo_f[d]) * lat.inv_f[d]) for d in range(5)]
        c = [min(int(math.floor(u[d])), int(lat.res[d]) - 2) for d in range(5)]
        inside = all(0 <= u[d] <= lat.res[d] - 1 for d in range(5))
        if not inside:
            assert ids[r] == -1
            continue
        lin = 0
        for d in range(5):
            lin = lin * (int(lat.res[d]) - 1) + c[d]
        assert ids[r] == lin


# ------------------------------------------------------------ classes fixed by geometry

def one_cell_map(lo, hi, nfit=64, seed=1):
    L = singlet()
    lat = oracle.Lattice([2, 2, 2, 2, 2], lo, hi)
    rng = np.random.default_rng(seed)
    q = rng.uniform(lo, hi, size=(nfit, 5))
    inv = 1 / np.sqrt(q[:, 2] ** 2 + q[:, 3] ** 2 + 1)
    f = np.float32
    rays = w.Rays(q[:, 0].astype(f), q[:, 1].astype(f), (q[:, 2] * inv).astype(f),
                  (q[:, 3] * inv).astype(f), inv.astype(f), q[:, 4].astype(f))
    return oracle.TableMap(L, (0, 0), lat, rays), rays


def test_cell_near_axis_is_valid():
    m, _ = one_cell_map([-1, -1, -0.01, -0.01, 500], [1, 1, 0.01, 0.01, 600])
    assert m.cell_class[0] == 1


def test_cell_beyond_the_stop_is_invalid():
    # every entrance point has r > 10.5 > stop radius 10
    m, _ = one_cell_map([10.5, -0.5, -0.05, -0.05, 400], [11.5, 0.5, 0.05, 0.05, 700])
    assert m.cell_class[0] == 0


def test_cell_across_the_stop_edge_is_boundary():
    m, _ = one_cell_map([9.0, -0.2, -0.01, -0.01, 500], [10.8, 0.2, 0.01, 0.01, 600])
    assert m.cell_class[0] == 2


# ------------------------------------------------------------ whole small map

@pytest.fixture(scope="module")
def small_map():
    L = singlet()
    lo, hi = box()
    lat = oracle.Lattice([6, 6, 6, 6, 3], lo, hi)
    rays = w.singlet_rays(4096)
    m = oracle.TableMap(L, (0, 0), lat, rays)
    return L, lat, rays, m


def test_query_classes_agree_with_exact_trace(small_map):
    L, lat, rays, m = small_map
    out, flags = m.query(rays)
    ex, ev, _, _ = L.trace(rays)
    fell_back = (flags & 16) != 0
    interp = (flags & 1 != 0) & ~fell_back
    # rays answered by the tracer are the tracer's answer, bit for bit
    assert np.array_equal(out[fell_back], ex[fell_back])
    assert np.array_equal(flags[fell_back] & 1, ev[fell_back] & 1)
    # rays in INVALID cells were fit rays there: all invalid in the exact trace
    invalid_cell = ((flags & 1) == 0) & ~fell_back
    assert np.all(ev[invalid_cell] == 0)
    # VALID cells: every fit ray inside was valid
    assert np.all(ev[interp] == 1)
    # interpolation of the coarse 6^4 x 3 lattice is close to the trace
    err = np.hypot(out[interp, 0] - ex[interp, 0], out[interp, 1] - ex[interp, 1])
    assert interp.sum() > 100
    assert np.max(err) < 1.0
    assert np.all(np.abs(np.linalg.norm(out[interp, 2:5], axis=1) - 1) < 1e-14)


def test_zero_residual_tolerance_makes_the_map_exact_on_fit_rays(small_map):
    L, lat, rays, m0 = small_map
    m = oracle.TableMap(L, (0, 0), lat, rays, tol=0.0)
    out, flags = m.query(rays)
    ex, ev, _, _ = L.trace(rays)
    assert np.array_equal(flags & 1, ev & 1)
    assert np.allclose(out, ex, atol=1e-12)
    assert (m.cell_class == 1).sum() <= (m0.cell_class == 1).sum()


def test_query_one_matches_whole_map(small_map):
    L, lat, rays, m = small_map
    out, flags = m.query(rays)
    ids = lat.cell_ids(rays)
    rng = np.random.default_rng(4)
    for r in rng.choice(len(rays), 60, replace=False):
        sel = np.nonzero(ids == ids[r])[0]
        fit = rays.subset(sel)
        ray = np.array([a[r] for a in rays.arrays()], np.float32)
        if ids[r] < 0:
            continue
        cell = lat.cell_of(ray)
        cls, corner6, cv, mr = oracle.classify_cell(L, (0, 0), lat, cell, fit)
        assert cls == m.cell_class[ids[r]]


# ---------------------------------------------------------------- 16-bit node table

def test_quantize16_round_trip_is_exact():
    """Values that are integer multiples of the chosen step come back
    unchanged: the step is a power of two, so value / step is exact and the
    rounding to an integer is the only rounding."""
    rng = np.random.default_rng(7)
    q = rng.integers(-32767, 32768, size=(5000, 6))
    q[0] = 32767            # the largest code sets the exponent: 2^14 <= 32767
    step = np.array([2.0 ** -10, 2.0 ** -15, 2.0 ** -16, 2.0 ** -3, 2.0 ** 0, 2.0 ** -20])
    v = q * step
    valid = np.ones(len(v), np.uint8)
    dec, steps = oracle.quantize16(v, valid)
    assert np.array_equal(steps, step)
    assert np.array_equal(dec, v)


def test_quantize16_error_bound_and_exponent():
    """|decoded - value| <= step / 2, and the step brackets the largest
    magnitude: 2^14 step <= max |v| < 2^15 step (so every code fits 16 bits);
    invalid nodes decode to zero whatever they held."""
    rng = np.random.default_rng(8)
    v = rng.normal(size=(20000, 6)) * np.array([17.0, 3.3, 0.21, 0.2, 0.97, 0.5])
    v[:, 4] = np.abs(v[:, 4])
    valid = (rng.uniform(size=len(v)) < 0.8).astype(np.uint8)
    dec, steps = oracle.quantize16(v, valid)
    ok = valid != 0
    m = np.abs(v[ok]).max(axis=0)
    assert np.all(2.0 ** 14 * steps <= m) and np.all(m < 2.0 ** 15 * steps)
    assert np.all(np.abs(dec[ok] - v[ok]) <= steps / 2)
    assert np.all(dec[~ok] == 0.0)
    # steps are powers of two
    assert np.all(np.frexp(steps)[0] == 0.5)


def test_quantized_map_query_within_half_a_step(small_map):
    """Multilinear interpolation is a convex combination of the 32 corners,
    so the quantised map's interpolated x, y and I stay within half a step of
    the FP64 map's (direction within a few steps after renormalisation);
    classes and traced rays are untouched."""
    L, lat, rays, m = small_map
    out0, f0 = m.query(rays)
    mq = oracle.TableMap(L, (0, 0), lat, rays)
    steps = mq.quantize16()
    out1, f1 = mq.query(rays)
    assert np.array_equal(f0, f1)
    interp = ((f1 & 1) != 0) & ((f1 & 16) == 0)
    assert interp.sum() > 100
    d = np.abs(out1[interp] - out0[interp])
    for k in (0, 1, 5):
        assert d[:, k].max() <= steps[k] / 2 * (1 + 1e-12)
    for k in (2, 3, 4):
        assert d[:, k].max() <= 4 * steps[2:5].max()
    traced = (f1 & 16) != 0
    assert np.array_equal(out1[traced], out0[traced])
