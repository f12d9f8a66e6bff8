"""GPU parity of the half-size node table (lt_build_map with LT_NODE_S16)
against the oracle's own map quantised by the same rule (oracle.quantize16):
the steps, the cell classes, and the query answers within the tracer's
tolerances plus one quantisation step.  One step is the right allowance: both
sides round their own node values (FP32 on the GPU, FP64 in the oracle) to
the nearest integer multiple of the same power of two, and two values a few
1e-7 apart can round to neighbouring integers.  Beside the oracle check, the
16-bit query is held to its FP32 twin on the GPU: the same classes and traced
rays bit for bit, interpolated x, y and I within half a step."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import DIR_TOL, EDGE_EPS, I_TOL, POS_TOL, TIR_EPS

pytestmark = pytest.mark.gpu

SMAX = math.tan(math.radians(10.0))


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


def gpu_query(gmap, rays, mode=lt.QUERY_TABLE):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    gmap.query(d.inp, d.lam, o.out, len(rays), mode)
    torch.cuda.synchronize()
    return o.numpy()


def corner_max(node_vals, res):
    k = node_vals.shape[1]
    m = node_vals.reshape(list(res) + [k])
    out = np.zeros([r - 1 for r in res] + [k])
    for c in range(32):
        b = [(c >> (4 - d)) & 1 for d in range(5)]
        out = np.maximum(out, m[tuple(slice(b[d], b[d] + res[d] - 1) for d in range(5))])
    return out.reshape(-1, k)


def half_step_check(o16, f16, o32, f32, steps, label):
    """The 16-bit query against the FP32 query of the same map on the GPU."""
    assert np.array_equal(f16, f32), f"{label}: flags differ between the node formats"
    traced = (f16 & lt.FLAG_TRACED) != 0
    assert np.array_equal(o16[traced].view(np.uint32), o32[traced].view(np.uint32)), f"{label}: traced rays differ"
    interp = ((f16 & lt.FLAG_VALID) != 0) & ~traced
    d = np.abs(o16[interp].astype(np.float64) - o32[interp])
    # half a step, plus FP32 rounding of the two interpolations (a few ulps of the value)
    ulp = 4 * np.spacing(np.abs(o32[interp]).astype(np.float32)).astype(np.float64)
    for k in (0, 1, 5):
        assert np.all(d[:, k] <= steps[k] / 2 + ulp[:, k]), f"{label}: output {k} beyond half a step"
    for k in (2, 3, 4):
        assert np.all(d[:, k] <= 4 * max(steps[2:5]) + 1e-6), f"{label}: direction {k}"
    return int(interp.sum()), d.max(axis=0) if len(d) else np.zeros(6)


def check_s16(presc, rho, fit, queries, res, label):
    lens, ol = lt.Lens(presc), oracle.Lens(presc)
    lo, hi = [-rho, -rho, -SMAX, -SMAX, 380.0], [rho, rho, SMAX, SMAX, 780.0]
    dfit = batch.DeviceRays(fit)
    g32 = lt.Map.build(lens, 0, res, lo, hi, fit=dfit)
    g16 = lt.Map.build(lens, 0, res, lo, hi, fit=dfit, node_format=lt.NODE_S16)
    s16, s32 = g16.stats(), g32.stats()
    assert s16["node_format"] == lt.NODE_S16 and s32["node_format"] == lt.NODE_F32
    N, NC = s16["n_nodes"], s16["n_cells"]
    assert s16["table_bytes"] < s32["table_bytes"] * 0.55
    steps = np.array(s16["node_step"], np.float64)

    n32, nv32, cc32 = g32.export(N, NC)
    n16, nv16, cc16 = g16.export(N, NC)
    assert np.array_equal(cc16, cc32) and np.array_equal(nv16, nv32)
    # the stored nodes are the FP32 nodes rounded to the step (half a step at most)
    ok = nv32 == 1
    assert np.all(np.abs(n16[ok].astype(np.float64) - n32[ok]) <= steps / 2)
    assert np.all(n16[~ok] == 0.0)

    # the oracle's map, quantised by the same rule, has the same steps
    lat = oracle.Lattice(res, lo, hi)
    omap = oracle.TableMap(ol, (0, 0), lat, fit)
    osteps = omap.quantize16()
    assert np.array_equal(osteps, steps), (label, osteps, steps)

    # queries against the oracle: same class -> within tolerance + one step
    gout, gfl = gpu_query(g16, queries)
    oout, ofl = omap.query(queries)
    qcells = lat.cell_ids(queries)
    same = np.ones(len(queries), bool)
    inside = qcells >= 0
    same[inside] = cc16[qcells[inside]] == omap.cell_class[qcells[inside]]
    interp = same & ((gfl & 0x10) == 0) & ((gfl & 1) != 0)
    assert np.array_equal(gfl[same] & 0x30, ofl[same] & 0x30), f"{label}: traced/outside flags differ"
    # nodes' own FP32 error against the FP64 trace, per cell (large only for
    # ill-conditioned corners): it reaches the interpolant through the corners
    nodes = lat.node_rays()
    ex, ev, edge, kmin = ol.trace(nodes)
    both = (nv32 == 1) & (ev == 1)
    nerr = np.zeros((N, 3))
    nerr[both, 0] = np.abs(n32[both, 0:2] - ex[both, 0:2]).max(axis=1)
    nerr[both, 1] = np.abs(n32[both, 2:5] - ex[both, 2:5]).max(axis=1)
    nerr[both, 2] = np.abs(n32[both, 5] - ex[both, 5])
    cerr = corner_max(nerr, res)[qcells[interp]]
    ep = np.abs(gout[interp, 0:2] - oout[interp, 0:2]).max(axis=1)
    ed = np.abs(gout[interp, 2:5] - oout[interp, 2:5]).max(axis=1)
    ei = np.abs(gout[interp, 5] - oout[interp, 5])
    assert np.all(ep <= POS_TOL + max(steps[0], steps[1]) + cerr[:, 0]), f"{label}: position"
    assert np.all(ed <= DIR_TOL + 4 * max(steps[2:5]) + cerr[:, 1]), f"{label}: direction"
    assert np.all(ei <= I_TOL + steps[5] + cerr[:, 2]), f"{label}: throughput"
    # the mask: bit-exact for rays of equal class, except flagged ones
    qex, qev, qedge, qkmin = ol.trace(queries)
    flagged = (qedge < EDGE_EPS) | (qkmin < TIR_EPS)
    mism = same & (((gfl & 1) != 0) != ((ofl & 1) != 0)) & ~flagged
    assert not mism.any(), f"{label}: {int(mism.sum())} unflagged validity mismatches"

    # against the FP32 twin on the GPU
    o32, f32 = gpu_query(g32, queries)
    n_int, dmax = half_step_check(gout, gfl, o32, f32, steps, label)
    print("s16", label, {"steps": steps.tolist(), "interpolated": n_int, "vs_f32_max": dmax.tolist(),
                         "vs_oracle_pos_max": float(ep.max()) if ep.size else 0.0,
                         "table_bytes": [s16["table_bytes"], s32["table_bytes"]]})
    assert n_int > 100
    return g16, g32


def test_singlet_s16():
    presc = w.singlet_lens()
    # even node counts on the slope axes: no node at slope 0, whose exit d_z
    # of exactly 1 would sit on a power of two (the steps' exponent boundary)
    check_s16(presc, 12.0, w.singlet_rays(6000), w.entrance_rays(20011, 31, 12.5),
              [9, 9, 8, 8, 4], "singlet")


def test_eleven_s16():
    presc = w.eleven_surface_lens(oracle_accept)
    rho = w.eleven_rho(presc)
    check_s16(presc, rho, w.entrance_rays(20000, 41, rho), w.entrance_rays(30011, 43, rho * 1.05),
              [8, 8, 8, 8, 3], "eleven")


def test_eleven_s16_full_size():
    """The headline lens at 32^4 x 8 from 16,777,216 fit rays, 4,194,304
    queries in the two-kernel form and a 65,536-ray batch in the one-kernel
    form: the 16-bit table against its FP32 twin, ray by ray."""
    presc = w.eleven_surface_lens(oracle_accept)
    lens = lt.Lens(presc)
    rho = w.eleven_rho(presc)
    lo, hi = [-rho, -rho, -SMAX, -SMAX, 380.0], [rho, rho, SMAX, SMAX, 780.0]
    fit = batch.DeviceRays(w.eleven_fit_rays(presc))
    g32 = lt.Map.build(lens, 0, [32, 32, 32, 32, 8], lo, hi, fit=fit)
    g16 = lt.Map.build(lens, 0, [32, 32, 32, 32, 8], lo, hi, fit=fit, node_format=lt.NODE_S16)
    del fit
    steps = np.array(g16.stats()["node_step"], np.float64)
    for n, seed in ((w.ELEVEN_N, w.SEED_BASE + 2), (65536, 77)):
        rays = w.entrance_rays(n, seed, rho)
        o16, f16 = gpu_query(g16, rays)
        o32, f32 = gpu_query(g32, rays)
        n_int, dmax = half_step_check(o16, f16, o32, f32, steps, f"eleven full {n}")
        print("s16 full", n, n_int, dmax.tolist())
        assert n_int > n // 10


def test_s16_no_mask_mode_and_noalloc():
    """LT_QUERY_NO_MASK interpolates every in-box ray (invalid nodes are
    zeros in both formats), and the allocation-free entry point gives the
    same bits as lt_query on a 16-bit map."""
    presc = w.singlet_lens()
    lens = lt.Lens(presc)
    lo, hi = [-12, -12, -SMAX, -SMAX, 380.0], [12, 12, SMAX, SMAX, 780.0]
    fit = batch.DeviceRays(w.singlet_rays(6000))
    g32 = lt.Map.build(lens, 0, [9, 9, 8, 8, 4], lo, hi, fit=fit)
    g16 = lt.Map.build(lens, 0, [9, 9, 8, 8, 4], lo, hi, fit=fit, node_format=lt.NODE_S16)
    steps = np.array(g16.stats()["node_step"], np.float64)
    rays = w.entrance_rays(5000, 9, 12.0)
    o16, f16 = gpu_query(g16, rays, lt.QUERY_NO_MASK)
    o32, f32 = gpu_query(g32, rays, lt.QUERY_NO_MASK)
    half_step_check(o16, f16, o32, f32, steps, "no mask")
    d = batch.DeviceRays(rays)
    a, b = batch.DeviceOut(len(rays)), batch.DeviceOut(len(rays))
    g16.query(d.inp, d.lam, a.out, len(rays))
    lt.query_noalloc(g16, d.inp, d.lam, b.out, len(rays))
    torch.cuda.synchronize()
    (oa, fa), (ob, fb) = a.numpy(), b.numpy()
    assert np.array_equal(oa.view(np.uint32), ob.view(np.uint32)) and np.array_equal(fa, fb)
    with pytest.raises(lt.LTError):
        g16.save("/tmp/should_not_exist.ltmap")
