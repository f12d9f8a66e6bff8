"""Pins of the oracle's polynomial-patch map (oracle/poly.py) against what the
paper and the mathematics fix, not against the oracle itself:

- a least-squares fit of total degree D reproduces every polynomial field of
  degree <= D exactly and no field of degree D + 1 (the term set and the
  patch-local coordinates are right);
- the symmetry reduction (Sec. 4.1, Eq. 10) is invariant under rotations
  about the axis and mirrors the tangential slope, and its rotation and
  mirror undo each other;
- apertures only decide validity: a ray valid through the real lens leaves
  the unclipped lens along exactly the same exit ray;
- classes rebuilt by brute force from freshly traced corner rays;
- the built map, queried on the workload's rays, stays within its certified
  residual of the exact FP64 trace (the tracer is the definition the map
  approximates; Sec. 4.2)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import poly
from paper_2605_04017_gb300 import workloads as w

SMAX = math.tan(math.radians(10.0)) * math.sqrt(2.0)


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def eleven():
    return w.eleven_surface_lens(oracle_accept)


def test_term_count():
    for D in range(6):
        assert len(poly.exponents(D)) == math.comb(D + 4, 4)
        assert all(sum(e) <= D for e in poly.exponents(D))


def _field(u, D, seed):
    """A polynomial field of total degree D in the reduced coordinates (5 outputs)."""
    rng = np.random.default_rng(seed)
    ctr = np.array([5.0, 0.0, 0.1, 4.0])
    scl = np.array([0.2, 5.0, 5.0, 0.3])
    z = (np.asarray(u, np.float64) - ctr) * scl
    out = np.zeros((len(z), 5))
    for k in range(5):
        acc = np.full(len(z), rng.uniform(-1, 1))
        for e in poly.exponents(D):
            if sum(e) == 0:
                continue
            acc = acc + rng.uniform(-0.3, 0.3) * np.prod([z[:, d] ** e[d] for d in range(4)], axis=0)
        out[:, k] = acc
    out[:, 2:4] *= 0.05          # direction components stay well inside the unit disc
    return out


@pytest.mark.parametrize("D", [2, 3, 4])
def test_polynomial_fields_reproduced_exactly(D):
    """Degree-D fields are fitted exactly; the map then returns them at any point of
    its patches (reduced frame: y = 0, q >= 0, so no rotation is involved)."""
    presc = w.singlet_lens()
    for deg_field, exact in ((D, True), (D + 1, False)):
        fn = lambda u: (_field(u, deg_field, 7), np.ones(len(u), bool))

        def node_fn(arrs):
            u, _, _, _ = poly.reduce_f64(*arrs)
            f = _field(u, deg_field, 7)
            out = np.zeros((len(u), 6))
            out[:, [0, 1, 2, 3, 5]] = f
            return out, np.ones(len(u), bool)

        pm = poly.PolyMap(presc, (0, 0), 12.0, SMAX, 380.0, 780.0, D, (2, 2, 1, 1), (2, 2, 2, 1),
                          D + 2, tol=1e-5, sample_fn=fn, node_fn=node_fn)
        rng = np.random.default_rng(3)
        u = np.stack([rng.uniform(0, 12, 500), rng.uniform(-SMAX, SMAX, 500),
                      rng.uniform(0, SMAX, 500), rng.uniform(1 / 0.78 ** 2, 1 / 0.38 ** 2, 500)], 1)
        G = pm.grid
        P = np.minimum(((u - G.lo) / G.h).astype(int), G.P - 1)
        pred = np.array([pm.evaluate(P[j], 2 * (u[j] - G.patch_lo(P[j])) / G.h - 1)[0] for j in range(len(u))])
        err = np.abs(pred - _field(u, deg_field, 7)).max()
        if exact:
            assert err < 1e-9, err
            assert np.all(pm.cell_class == poly.CELL_VALID)
        else:
            assert err > 1e-6, err
            assert np.any(pm.cell_class == poly.CELL_BOUNDARY)


def _rotate(rays, ang, mirror=False):
    x, y, dx, dy, dz, lam = (np.asarray(a, np.float64) for a in rays.arrays())
    if mirror:
        y, dy = -y, -dy
    c, s = math.cos(ang), math.sin(ang)
    return (c * x - s * y, s * x + c * y, c * dx - s * dy, s * dx + c * dy, dz, lam)


def test_reduction_invariant_under_rotation_and_mirror():
    rays = w.entrance_rays(4000, 11, 12.0)
    u0, c0, s0, m0 = poly.reduce_f64(*[np.asarray(a, np.float64) for a in rays.arrays()])
    for ang in (0.3, 1.9, -2.7):
        u1, _, _, m1 = poly.reduce_f64(*_rotate(rays, ang))
        assert np.abs(u1 - u0).max() < 1e-12
        assert np.array_equal(m1, m0)
    u2, _, _, m2 = poly.reduce_f64(*_rotate(rays, 0.0, mirror=True))
    assert np.abs(u2 - u0).max() < 1e-12
    nz = u0[:, 2] > 1e-12
    assert np.array_equal(m2[nz], -m0[nz])


def test_reduction_round_trip():
    """Rotating the reduced ray back by (c, s) after the mirror restores the input."""
    rays = w.entrance_rays(4000, 12, 12.0)
    x, y, dx, dy, dz, lam = (np.asarray(a, np.float64) for a in rays.arrays())
    u, c, s, m = poly.reduce_f64(x, y, dx, dy, dz, lam)
    r, p, q, wv = u.T
    assert np.abs(c * r - x).max() < 1e-12 and np.abs(s * r - y).max() < 1e-12
    assert np.abs((c * p - s * m * q) - dx / dz).max() < 1e-12
    assert np.abs((s * p + c * m * q) - dy / dz).max() < 1e-12
    assert np.abs(wv - (1000.0 / lam) ** 2).max() < 1e-12
    # the reduced ray of u is the ray rotated onto +x with d_y >= 0
    rr = poly.reduced_rays_f64(u)
    assert np.abs(rr[2] / rr[4] - p).max() < 1e-12 and np.abs(rr[3] / rr[4] - q).max() < 1e-12


def test_fp32_rule_close_to_fp64():
    rays = w.entrance_rays(20000, 13, 12.0)
    u32, ok = poly.reduce_f32(*rays.arrays())
    u64, _, _, _ = poly.reduce_f64(*[np.asarray(a, np.float64) for a in rays.arrays()])
    assert ok.all()
    scale = np.array([12.0, 0.25, 0.25, 7.0])
    assert np.all(np.abs(u32 - u64) <= 8 * np.finfo(np.float32).eps * scale)


def test_fp32_node_rays_sit_on_their_nodes():
    G = poly.PolyGrid(12.0, SMAX, 380.0, 780.0, (2, 2, 1, 1), (3, 3, 4, 2))
    idx = np.array(list(np.ndindex(*G.node_shape())))
    arrs = G.node_rays_f32(idx)
    u, _, _, _ = poly.reduce_f64(*[np.asarray(a, np.float64) for a in arrs])
    nominal = G.lo + idx * (G.hi - G.lo) / G.C
    scale = np.array([12.0, 0.25, 0.25, 7.0])
    assert np.all(np.abs(u - nominal) <= 16 * np.finfo(np.float32).eps * scale)


def test_unclipped_lens_agrees_on_valid_rays(eleven):
    rays = w.eleven_rays(eleven, 30000)
    real = oracle.Lens(eleven)
    openl = oracle.Lens(poly.unclipped(eleven))
    for path in [(0, 0), oracle.path_ij(11, 17)]:
        o1, v1, _, _ = real.trace(rays, path)
        o2, v2, _, _ = openl.trace(rays, path)
        ok = v1 == 1
        assert ok.sum() > 100
        assert np.all(v2[ok] == 1)
        assert np.array_equal(o1[ok], o2[ok])
        # vignetting is real: some rays lost by the lens pass the unclipped one
        assert np.sum((v1 != 1) & (v2 == 1)) > 100


@pytest.fixture(scope="module")
def singlet_map():
    presc = w.singlet_lens()
    fit = w.entrance_rays(20000, 21, 12.0)
    return poly.PolyMap(presc, (0, 0), 12.0, SMAX, 380.0, 780.0, 4, (8, 8, 4, 1), (2, 2, 2, 2), 6,
                        tol=1e-4, fit_rays=fit)


@pytest.fixture(scope="module")
def eleven_map(eleven):
    rho = w.eleven_rho(eleven)
    return poly.PolyMap(eleven, (0, 0), rho, SMAX, 380.0, 780.0, 4, (4, 4, 2, 1), (4, 4, 4, 4), 6,
                        tol=1e-4)


def test_brute_force_classes(singlet_map):
    """A cell's class from its 16 corner rays traced afresh, one by one."""
    pm = singlet_map
    rng = np.random.default_rng(5)
    cells = [tuple(rng.integers(0, pm.grid.C)) for _ in range(60)]
    cells += [tuple(c) for c in np.argwhere(pm.cell_class == poly.CELL_BOUNDARY)[:20]]
    for cell in cells:
        corners = list(itertools.product((0, 1), repeat=4))
        idx = np.array([np.asarray(cell) + k for k in corners])
        arrs = pm.grid.node_rays_f32(idx)
        vs, outs = [], []
        for j in range(16):
            v, o, _, _ = pm.lens.trace_one(*[a[j] for a in arrs], path=(0, 0))
            vs.append(v == 1)
            outs.append(o)
        if not any(vs):
            want = poly.CELL_INVALID
        elif not all(vs):
            want = poly.CELL_BOUNDARY
        else:
            P = np.asarray(cell) // pm.grid.m
            xi = np.array([2.0 * (np.asarray(cell) + k - P * pm.grid.m) / pm.grid.m - 1 for k in corners])
            pred = pm.evaluate(P, xi)
            o = np.array(outs)
            res = np.hypot(pred[:, 0] - o[:, 0], pred[:, 1] - o[:, 1]).max()
            want = poly.CELL_VALID if res <= pm.tol else poly.CELL_BOUNDARY
        built = pm.cell_class[cell]
        # fit rays may only demote a cell to BOUNDARY
        assert built == want or built == poly.CELL_BOUNDARY, (cell, built, want)


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_map_within_certified_residual_of_exact_trace(which, singlet_map, eleven_map, eleven):
    if which == "singlet":
        pm, rays = singlet_map, w.singlet_rays(30000)
    else:
        pm, rays = eleven_map, w.eleven_rays(eleven, 30000)
    out, flags = pm.query(rays)
    ex, ev, edge, _ = pm.lens.trace(rays, (0, 0))
    interp = (flags & 1 != 0) & (flags & 16 == 0)
    traced = flags & 16 != 0
    assert interp.sum() > 0.7 * np.sum(ev == 1)
    # the mask: interpolated rays are valid, rays of INVALID cells are invalid
    clear = edge > 1e-6
    assert np.all(ev[interp & clear] == 1)
    assert np.all(ev[(flags == 0) & clear] != 1)
    # traced rays are the exact trace
    assert np.array_equal(out[traced], ex[traced])
    e_pos = np.abs(out[interp, :2] - ex[interp, :2]).max()
    e_dir = np.abs(out[interp, 2:5] - ex[interp, 2:5]).max()
    e_I = np.abs(out[interp, 5] - ex[interp, 5]).max()
    print(which, "interpolated", interp.mean(), "traced", traced.mean(), "pos", e_pos, "dir", e_dir, "I", e_I)
    assert e_pos <= 1e-4
    assert e_dir <= 1e-5 and e_I <= 1e-5
    # rotating every input rotates every output (Sec. 4.1, Eq. 10)
    rot = w.Rays(*[np.asarray(a, np.float32) for a in _rotate(rays, 0.9)])
    out2, flags2 = pm.query(rot)
    both = (flags & 1 != 0) & (flags2 & 1 != 0) & (flags & 16 == 0) & (flags2 & 16 == 0)
    c, s = math.cos(0.9), math.sin(0.9)
    want_x = c * out[both, 0] - s * out[both, 1]
    want_dx = c * out[both, 2] - s * out[both, 3]
    assert np.abs(out2[both, 0] - want_x).max() < 2e-4
    assert np.abs(out2[both, 2] - want_dx).max() < 2e-5


def test_no_mask_ablation(singlet_map):
    """Without the mask every ray inside the box gets the regressor's answer."""
    rays = w.singlet_rays(5000)
    out, flags = singlet_map.query(rays, use_mask=False)
    inside = flags & 32 == 0
    assert np.all(flags[inside] & 1 == 1)
    ex, ev, _, _ = singlet_map.lens.trace(rays, (0, 0))
    # vignetted rays now get an output although the lens stops them
    assert np.sum((ev != 1) & (flags & 1 == 1)) > 100


def test_fresh_classes_match_the_table(singlet_map):
    """classify_fresh (a cell's corners traced afresh plus its fit rays) agrees
    with the class table built in one pass."""
    pm = singlet_map
    rng = np.random.default_rng(8)
    cells = [tuple(rng.integers(0, pm.grid.C)) for _ in range(80)]
    cells += [tuple(c) for c in np.argwhere(pm.cell_class == poly.CELL_BOUNDARY)[:20]]
    for cell in cells:
        assert pm.classify_fresh(cell)[0] == pm.cell_class[cell], cell


def test_batched_classes_match_fresh(singlet_map):
    """classify_cells (many cells in one pass) agrees with classify_fresh cell by cell."""
    pm = singlet_map
    rng = np.random.default_rng(9)
    cells = np.array([rng.integers(0, pm.grid.C) for _ in range(120)])
    cells = np.concatenate([cells, np.argwhere(pm.cell_class == poly.CELL_BOUNDARY)[:30]])
    cls, res = pm.classify_cells(cells)
    for j, c in enumerate(cells):
        want, wres = pm.classify_fresh(tuple(c))
        assert cls[j] == want, (c, cls[j], want)
        assert abs(res[j] - wres) <= 1e-12 * max(1.0, wres)
