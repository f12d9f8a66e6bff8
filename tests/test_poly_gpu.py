"""GPU parity of the polynomial-patch map (lt_build_poly_map, lt_query) against
the oracle's own map (oracle/poly.py), through the C ABI:

- the fit: every patch's polynomial against the oracle's FP64 fit (the GPU
  traces its samples in FP32 and solves FP64 normal equations);
- the mask: node validity and cell classes, differing only where a corner
  ray passes within 1e-6 mm of an aperture edge or a residual sits at the
  certification threshold;
- queries element by element: polynomial answers within the tracer's own
  tolerances of the oracle's, traced answers by the tracer's parity rule;
- the large-batch (queue) form against the one-kernel form, bit for bit, and
  the allocation-free entry point on such a map;
- the full-size 11-surface workload: sampled parity against cells the
  oracle classifies afresh, and every ray against the FP32 trace at the
  metric's 1e-4 mm."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import poly
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import DIR_TOL, I_TOL, POS_TOL, compare_trace

pytestmark = pytest.mark.gpu

SMAX = math.tan(math.radians(10.0)) * math.sqrt(2.0)
EDGE = 1e-6
F_VALID, F_BAD, F_TRACED, F_OUTSIDE = 1, 8, 0x10, 0x20


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def eleven():
    return w.eleven_surface_lens(oracle_accept)


def gpu_query(gmap, rays, mode=lt.QUERY_TABLE):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    gmap.query(d.inp, d.lam, o.out, len(rays), mode)
    torch.cuda.synchronize()
    return o.numpy()


def build_pair(presc, rho, cfg, fit):
    lens = lt.Lens(presc)
    g = lt.Map.build_poly(lens, 0, rho, SMAX, cfg["degree"], cfg["patches"], cfg["cells"], cfg["samples"],
                          fit=batch.DeviceRays(fit) if fit is not None else None,
                          max_residual_mm=cfg["tol"])
    o = poly.PolyMap(presc, (0, 0), rho, SMAX, 380.0, 780.0, cfg["degree"], cfg["patches"], cfg["cells"],
                     cfg["samples"], tol=cfg["tol"], fit_rays=fit)
    return lens, g, o


SINGLET_CFG = dict(degree=4, patches=(8, 8, 4, 1), cells=(2, 2, 2, 2), samples=6, tol=1e-4)
ELEVEN_CFG = dict(degree=3, patches=(8, 8, 4, 2), cells=(2, 2, 2, 2), samples=5, tol=1e-4)


@pytest.fixture(scope="module")
def singlet_pair():
    fit = w.entrance_rays(20000, 21, 12.0)
    return build_pair(w.singlet_lens(), 12.0, SINGLET_CFG, fit)


@pytest.fixture(scope="module")
def eleven_pair(eleven):
    fit = w.entrance_rays(50000, 22, w.eleven_rho(eleven))
    return build_pair(eleven, w.eleven_rho(eleven), ELEVEN_CFG, fit)


def _eval(coef_p, exps, xi):
    X = np.stack([np.prod([xi[:, k] ** e[k] for k in range(4)], axis=0) for e in exps], 1)
    return X @ coef_p


def _samples(o):
    """The fit's sample rays, computed as the library computes them (FP64, each
    operation rounded once, then rounded to FP32), patch by patch."""
    G = o.grid
    ns = round(len(o.xi_s) ** 0.25)
    cheb = [math.cos(math.pi * (j + 0.5) / ns) for j in range(ns)]
    lo = G.lo
    h = (G.hi - G.lo) / G.P
    rays = []
    for pid in range(G.n_patches):
        pk = np.array(np.unravel_index(pid, tuple(G.P)), np.float64)
        idx = np.array(list(np.ndindex(ns, ns, ns, ns)))
        u = np.stack([lo[k] + (pk[k] + 0.5 * (np.array(cheb)[idx[:, k]] + 1.0)) * h[k] for k in range(4)], 1)
        inv = 1.0 / np.sqrt((u[:, 1] * u[:, 1] + u[:, 2] * u[:, 2]) + 1.0)
        rays.append(np.stack([u[:, 0], np.zeros(len(u)), u[:, 1] * inv, u[:, 2] * inv, inv,
                              1000.0 / np.sqrt(u[:, 3])], 1))
    a = np.concatenate(rays).astype(np.float32)
    return w.Rays(*[np.ascontiguousarray(a[:, k]) for k in range(6)])


def _gpu_unclipped(presc):
    """The prescription with every aperture opened to the edge of its sphere's
    near cap and no stop (the library's own build removes them outright; a
    ray reaching past 0.9999999 of a sphere's radius does not occur)."""
    import copy
    U = copy.deepcopy(presc)
    for s in U.surfaces:
        s.aperture_r = 0.9999999 / abs(s.curvature) if s.curvature != 0 else 1e6
    U.stop_r = 0.0
    return U


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_fit_matches_oracle(which, singlet_pair, eleven_pair, eleven):
    """The fit is linear in its samples, so the GPU's and the oracle's fits
    differ exactly by the least-squares image of their sample traces'
    differences.  Checked as (1) the GPU's FP32 traces of the sample rays
    against the oracle's FP64 ones, by the tracer's parity rule, and (2) the
    GPU's coefficients against an FP64 least-squares fit of those same GPU
    traces (the normal-equation reductions and the Cholesky solve)."""
    presc = w.singlet_lens() if which == "singlet" else eleven
    _, g, o = singlet_pair if which == "singlet" else eleven_pair
    coef, exps, ok = g.poly_export()
    ps = g.poly_stats()
    assert ps["patches"] == o.grid.n_patches and ps["terms"] == len(o.exps)
    assert sorted(map(tuple, exps)) == sorted(o.exps)
    samples = _samples(o)
    M = len(o.xi_s)
    assert ps["samples_traced"] == len(samples)
    d = batch.DeviceRays(samples)
    t = batch.DeviceOut(len(samples))
    lt.trace(lt.Lens(_gpu_unclipped(presc)), d.inp, d.lam, 0, t.out, len(samples))
    torch.cuda.synchronize()
    gout, gfl = t.numpy()
    ex, ev, edge, kmin = o.open.trace(samples, (0, 0))
    st = compare_trace(gout, gfl, ex, ev, None, kmin, f"{which} fit samples",
                       cond=(o.open, samples, (0, 0)), max_exempt_frac=0.02)
    assert ps["samples_valid"] == int((gfl & F_VALID).sum())
    # (2) FP64 least squares of the GPU's own traces, in the library's term order
    A = np.stack([np.prod([o.xi_s[:, k] ** e[k] for k in range(4)], axis=0) for e in exps], 1)
    gv = (gfl & F_VALID != 0).reshape(o.grid.n_patches, M)
    gy = gout[:, [0, 1, 2, 3, 5]].astype(np.float64).reshape(o.grid.n_patches, M, 5)
    worst = np.zeros(5)
    xi = np.random.default_rng(1).uniform(-1, 1, (300, 4))
    X = np.stack([np.prod([xi[:, k] ** e[k] for k in range(4)], axis=0) for e in exps], 1)
    for pid in range(o.grid.n_patches):
        fit_ok = gv[pid].sum() >= len(exps) and np.linalg.matrix_rank(A[gv[pid]]) == len(exps)
        assert bool(ok[pid]) == fit_ok, pid
        if not fit_ok:
            continue
        c, *_ = np.linalg.lstsq(A[gv[pid]], gy[pid][gv[pid]], rcond=None)
        worst = np.maximum(worst, np.abs(X @ coef[pid] - X @ c).max(axis=0))
    print(which, "GPU fit vs FP64 least squares of its samples:", worst, "stats", ps,
          "samples exempt", st["exempt"])
    assert worst[:2].max() <= 1e-6 and worst[2:].max() <= 1e-8


def _node_edges(o):
    """Oracle edge distance of every class-grid node ray (node order)."""
    idx = np.array(list(np.ndindex(*o.grid.node_shape())))
    arrs = o.grid.node_rays_f32(idx)
    _, _, edge, _ = o.lens.trace(w.Rays(*arrs), o.path)
    return edge.reshape(o.grid.node_shape())


def _explained_cells(o, node_edge, cells, fit=None):
    """Cells whose class may differ between FP32 and FP64 builds: a corner ray or
    a fit ray of the cell within EDGE of an aperture edge, or a residual at the
    certification threshold."""
    import itertools
    corners = np.array(list(itertools.product((0, 1), repeat=4)))
    near = set()
    if fit is not None:
        inside, fc = o.locate(fit)
        _, _, fe, _ = o.lens.trace(fit, o.path)
        for r in np.nonzero(inside & (fe < EDGE))[0]:
            near.add(tuple(fc[r]))
    out = []
    for c in cells:
        c = tuple(int(v) for v in c)
        ne = any(node_edge[tuple(np.asarray(c) + k)] < EDGE for k in corners)
        border = abs(o.cell_res[c] - o.tol) <= 2e-5
        out.append(ne or border or c in near)
    return np.array(out, bool)


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_mask_matches_oracle(which, singlet_pair, eleven_pair):
    _, g, o = singlet_pair if which == "singlet" else eleven_pair
    nn, nc = o.grid.node_shape(), tuple(int(c) for c in o.grid.C)
    nv, cc = g.export_mask(int(np.prod(nn)), int(np.prod(nc)))
    node_edge = _node_edges(o)
    dv = nv.reshape(nn).astype(bool) != o.node_valid
    assert np.all(node_edge[dv] < EDGE), "node validity differs away from an aperture edge"
    cc = cc.reshape(nc)
    dc = np.argwhere(cc != o.cell_class)
    fit = w.entrance_rays(20000, 21, 12.0) if which == "singlet" else None
    ok = _explained_cells(o, node_edge, dc, fit) if len(dc) else np.ones(0, bool)
    print(which, "node mismatches", int(dv.sum()), "cell mismatches", len(dc), "unexplained", int((~ok).sum()),
          "classes", np.bincount(cc.ravel(), minlength=3))
    assert ok.all(), dc[~ok][:10]


def _compare_queries(gout, gflags, oout, oflags, o, rays, label):
    g_int = (gflags & F_VALID != 0) & (gflags & F_TRACED == 0)
    o_int = (oflags & F_VALID != 0) & (oflags & F_TRACED == 0)
    g_tr, o_tr = gflags & F_TRACED != 0, oflags & F_TRACED != 0
    assert np.array_equal(gflags & F_BAD != 0, oflags & F_BAD != 0), label
    assert np.array_equal(gflags & F_OUTSIDE != 0, oflags & F_OUTSIDE != 0), label
    both = g_int & o_int
    dp = np.abs(gout[both, :2].astype(np.float64) - oout[both, :2]).max(initial=0.0)
    dd = np.abs(gout[both, 2:5].astype(np.float64) - oout[both, 2:5]).max(initial=0.0)
    di = np.abs(gout[both, 5].astype(np.float64) - oout[both, 5]).max(initial=0.0)
    # rays the two sides answer differently sit in cells classed differently
    diff = (g_int != o_int) | (g_tr != o_tr)
    st = {"label": label, "interpolated": int(both.sum()), "traced": int((g_tr & o_tr).sum()),
          "class_differs": int(diff.sum()), "pos": dp, "dir": dd, "I": di}
    print("poly parity", st)
    assert dp <= POS_TOL and dd <= DIR_TOL and di <= I_TOL, st
    # rays of INVALID cells on both sides: no output
    inv = (gflags == 0) & (oflags == 0)
    assert np.all(gout[inv] == 0.0)
    # traced on both sides: the tracer's parity rule
    bt = g_tr & o_tr
    if bt.any():
        ex, ev, edge, kmin = o.lens.trace(rays.subset(np.nonzero(bt)[0]), o.path)
        compare_trace(gout[bt], gflags[bt] & ~np.uint8(F_TRACED | F_OUTSIDE), ex, ev, edge, kmin,
                      label + " traced", cond=(o.lens, rays.subset(np.nonzero(bt)[0]), o.path))
    return diff


def test_singlet_query_matches_oracle(singlet_pair):
    lens, g, o = singlet_pair
    rays = w.singlet_rays()                      # all 65,536 rays (one-kernel form)
    gout, gflags = gpu_query(g, rays)
    oout, oflags = o.query(rays)
    diff = _compare_queries(gout, gflags, oout, oflags, o, rays, "singlet")
    if diff.any():
        _, cells = o.locate(rays)
        ok = _explained_cells(o, _node_edges(o), cells[diff], w.entrance_rays(20000, 21, 12.0))
        assert ok.all()


def test_singlet_no_mask_matches_oracle(singlet_pair):
    lens, g, o = singlet_pair
    rays = w.singlet_rays(20000)
    gout, gflags = gpu_query(g, rays, lt.QUERY_NO_MASK)
    oout, oflags = o.query(rays, use_mask=False)
    _compare_queries(gout, gflags, oout, oflags, o, rays, "singlet no mask")


def test_bad_and_ragged_inputs(singlet_pair):
    lens, g, o = singlet_pair
    rays = w.singlet_rays(1001)
    rays.x[3] = np.nan
    rays.dz[5] = -0.5
    rays.lam[7] = 0.0
    rays.x[9] = 1e9                               # outside the box: traced (and lost)
    gout, gflags = gpu_query(g, rays)
    oout, oflags = o.query(rays)
    _compare_queries(gout, gflags, oout, oflags, o, rays, "singlet bad inputs")
    assert gflags[3] & F_BAD and gflags[5] & F_BAD and gflags[7] & F_BAD
    assert gflags[9] & F_OUTSIDE
    # n = 0 is a no-op
    d = batch.DeviceRays(rays)
    out = batch.DeviceOut(1)
    g.query(d.inp, d.lam, out.out, 0)
    torch.cuda.synchronize()


def test_eleven_query_matches_oracle(eleven_pair, eleven):
    lens, g, o = eleven_pair
    rays = w.eleven_rays(eleven, 40000)
    gout, gflags = gpu_query(g, rays)
    oout, oflags = o.query(rays)
    diff = _compare_queries(gout, gflags, oout, oflags, o, rays, "eleven")
    if diff.any():
        _, cells = o.locate(rays)
        ok = _explained_cells(o, _node_edges(o), cells[diff], w.entrance_rays(50000, 22, w.eleven_rho(eleven)))
        assert ok.all()


def test_queue_form_equals_one_kernel_form(eleven_pair, eleven):
    """A batch above 2^18 rays runs as the query kernel plus the queue tracer;
    the same rays in chunks of at most 2^18 run as one kernel: bit for bit."""
    lens, g, o = eleven_pair
    n = (1 << 19) + 12345
    rays = w.eleven_rays(eleven, n)
    big_out, big_flags = gpu_query(g, rays)
    d = batch.DeviceRays(rays)
    o2 = batch.DeviceOut(n)
    step = 1 << 18
    for a in range(0, n, step):
        b = min(n, a + step)
        g.query([t[a:b] for t in d.inp], d.lam[a:b], [t[a:b] for t in o2.out], b - a)
    torch.cuda.synchronize()
    small_out, small_flags = o2.numpy()
    assert np.array_equal(big_flags, small_flags)
    assert np.array_equal(big_out.view(np.uint32), small_out.view(np.uint32))
    # the allocation-free entry point gives the same answers on this kind of map
    m = 1 << 19
    o3 = batch.DeviceOut(m)
    lt.query_noalloc(g, [t[:m] for t in d.inp], d.lam[:m], o3.out, m)
    torch.cuda.synchronize()
    na_out, na_flags = o3.numpy()
    assert np.array_equal(na_flags, big_flags[:m])
    assert np.array_equal(na_out.view(np.uint32), big_out[:m].view(np.uint32))
    # the host entry point, pinned and pageable arrays
    for pin in (True, False):
        h = batch.HostRays(rays, pin=pin)
        g.query_host(h.inp[:5], h.inp[5], h.out + [h.flags], n)
        assert np.array_equal(h.flags.numpy(), big_flags), pin
        assert np.array_equal(np.stack([t.numpy() for t in h.out], 1).view(np.uint32), big_out.view(np.uint32)), pin


FULL_CFG = dict(degree=4, patches=(8, 8, 4, 1), cells=(16, 16, 16, 8), samples=6, tol=1e-4)


def test_eleven_full_size(eleven):
    """The headline workload: 4,194,304 rays of the 11-surface lens, the map
    fitted with the 16,777,216 fit rays.  Every ray against the FP32 trace at
    the metric's 1e-4 mm; 4,096 sampled rays against the oracle, whose cells
    it classifies afresh."""
    rho = w.eleven_rho(eleven)
    fit = w.eleven_fit_rays(eleven)
    lens = lt.Lens(eleven)
    cfg = FULL_CFG
    g = lt.Map.build_poly(lens, 0, rho, SMAX, cfg["degree"], cfg["patches"], cfg["cells"], cfg["samples"],
                          fit=batch.DeviceRays(fit), max_residual_mm=cfg["tol"])
    print("full-size map", g.stats(), g.poly_stats())
    rays = w.eleven_rays(eleven)
    gout, gflags = gpu_query(g, rays)
    d = batch.DeviceRays(rays)
    t = batch.DeviceOut(len(rays))
    lt.trace(lens, d.inp, d.lam, 0, t.out, len(rays))
    torch.cuda.synchronize()
    tout, tflags = t.numpy()
    interp = (gflags & F_VALID != 0) & (gflags & F_TRACED == 0)
    err = np.abs(gout[interp, :2].astype(np.float64) - tout[interp, :2]).max(axis=1)
    derr = np.abs(gout[interp, 2:5].astype(np.float64) - tout[interp, 2:5]).max()
    mism = (gflags & F_VALID != 0) != (tflags & F_VALID != 0)
    print("vs FP32 trace: interpolated", interp.mean(), "traced", (gflags & F_TRACED != 0).mean(),
          "pos max", err.max(), "p99", np.percentile(err, 99), "dir max", derr,
          "validity mismatches", int(mism.sum()), "of which near an edge", int((mism & (tflags & 2 != 0)).sum()))
    assert np.all(tflags[interp] & F_VALID)
    assert err.max() <= 1e-4
    assert mism.sum() <= 1e-5 * len(rays)
    # sampled oracle parity
    o = poly.PolyMap(eleven, (0, 0), rho, SMAX, 380.0, 780.0, cfg["degree"], cfg["patches"], cfg["cells"],
                     cfg["samples"], tol=cfg["tol"], fit_rays=fit, build_mask=False)
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(len(rays), 4096, replace=False))
    sub = rays.subset(idx)
    inside, cells = o.locate(sub)
    classes = np.full(len(idx), poly.CELL_BOUNDARY, np.uint8)
    res = np.zeros(len(idx))
    for j in np.nonzero(inside)[0]:
        classes[j], res[j] = o.classify_fresh(cells[j])
    oout, oflags = o.query(sub, classes=classes)
    diff = _compare_queries(gout[idx], gflags[idx], oout, oflags, o, sub, "eleven full size sampled")
    # a class decided differently: a corner within 1e-6 mm of an edge or a residual at the threshold
    for j in np.nonzero(diff)[0]:
        import itertools
        corners = np.array(list(itertools.product((0, 1), repeat=4)))
        arrs = o.grid.node_rays_f32(cells[j] + corners)
        _, _, e, _ = o.lens.trace(w.Rays(*arrs), o.path)
        assert e.min() < EDGE or abs(res[j] - cfg["tol"]) <= 2e-5, (j, cells[j], res[j])
