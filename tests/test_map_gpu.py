"""GPU parity of the tabulated map (lt_build_map / lt_query) against the
oracle's own map of the same lens, lattice and fit rays: node tables, cell
classes and query answers, at the full sizes of both workloads (singlet:
32^4 x 8 lattice fitted and queried on its 65,536 rays; 11-surface lens:
32^4 x 8 lattice fitted from 16,777,216 rays, 4,194,304 queries)."""
import math
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import (DIR_TOL, EDGE_EPS, GRAZING_K, I_TOL, POS_TOL, TIR_EPS, compare_trace)

pytestmark = pytest.mark.gpu

SMAX = math.tan(math.radians(10.0))
RES = [32, 32, 32, 32, 8]


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


def box(rho):
    return [-rho, -rho, -SMAX, -SMAX, 380.0], [rho, rho, SMAX, SMAX, 780.0]


def any_corner(node_mask, res):
    """Per cell (table order): does any of its 32 corner nodes have node_mask set?"""
    m = node_mask.reshape(res)
    out = np.zeros([r - 1 for r in res], bool)
    for k in range(32):
        b = [(k >> (4 - d)) & 1 for d in range(5)]
        out |= m[tuple(slice(b[d], b[d] + res[d] - 1) for d in range(5))]
    return out.reshape(-1)


def corner_max(node_vals, res):
    """Per cell (table order): the largest value of node_vals [N, k] over its 32 corners."""
    k = node_vals.shape[1]
    m = node_vals.reshape(list(res) + [k])
    out = np.zeros([r - 1 for r in res] + [k])
    for c in range(32):
        b = [(c >> (4 - d)) & 1 for d in range(5)]
        out = np.maximum(out, m[tuple(slice(b[d], b[d] + res[d] - 1) for d in range(5))])
    return out.reshape(-1, k)


def gpu_query(gmap, rays, mode=lt.QUERY_TABLE):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    gmap.query(d.inp, d.lam, o.out, len(rays), mode)
    torch.cuda.synchronize()
    return o.numpy()


def check_map(presc, rho, fit, queries, res=RES, label="", lens=None, ol=None, smax=SMAX):
    """lens / ol: the library's and the oracle's lens when they are not built
    from `presc` (the reversed lens of the backward map)."""
    lens = lens or lt.Lens(presc)
    ol = ol or oracle.Lens(presc)
    lo, hi = [-rho, -rho, -smax, -smax, 380.0], [rho, rho, smax, smax, 780.0]
    dfit = batch.DeviceRays(fit)
    gmap = lt.Map.build(lens, 0, res, lo, hi, fit=dfit)
    st = gmap.stats()
    lat = oracle.Lattice(res, lo, hi)
    omap = oracle.TableMap(ol, (0, 0), lat, fit)
    N, NC = lat.n_nodes, lat.n_cells
    assert st["n_nodes"] == N and st["n_cells"] == NC
    node6, nv, cc = gmap.export(N, NC)

    # ---- nodes: traced exactly; compare like any trace
    nodes = lat.node_rays()
    ex, ev, edge, kmin = ol.trace(nodes)
    assert np.array_equal(ev == 1, omap.node_valid == 1)
    flags = nv.astype(np.uint8)          # node records carry validity only
    node_st = compare_trace(node6, flags, ex, ev, edge, kmin, f"{label} nodes",
                            cond=(ol, nodes, (0, 0)))

    # ---- cells: classes equal except where a corner or fit ray is near an edge/TIR
    node_amb = (edge < EDGE_EPS) | (kmin < TIR_EPS)
    node_ill = kmin < GRAZING_K
    fex, fev, fedge, fkmin = ol.trace(fit)
    fit_amb = (fedge < EDGE_EPS) | (fkmin < TIR_EPS)
    fit_cells = lat.cell_ids(fit)
    amb_cells = set(fit_cells[fit_amb & (fit_cells >= 0)].tolist())
    mism = np.nonzero(cc != omap.cell_class)[0]
    cell_amb = any_corner(node_amb, res)
    for cid in mism:
        assert int(cid) in amb_cells or cell_amb[cid], \
            f"{label}: cell {cid} class {cc[cid]} vs oracle {omap.cell_class[cid]}"
    counts = np.bincount(cc, minlength=3)
    assert counts[0] == st["cells_invalid"] and counts[1] == st["cells_valid"]

    # ---- queries: same class -> same answer within the trace tolerances
    gout, gfl = gpu_query(gmap, queries)
    oout, ofl = omap.query(queries)
    qcells = lat.cell_ids(queries)
    same = np.ones(len(queries), bool)
    inside = qcells >= 0
    same[inside] = cc[qcells[inside]] == omap.cell_class[qcells[inside]]
    assert np.array_equal(gfl[same] & 0x30, ofl[same] & 0x30), f"{label}: traced/outside flags differ"
    # Interpolated rays of a cell with an ill-conditioned corner: the interpolant
    # mixes the 32 corner records, so its error is bounded by the largest
    # corner error the node comparison above certified, plus the tolerance
    # (FP32 interpolation rounding).  Every other ray goes through the
    # tracer's parity rule.
    cell_ill = any_corner(node_ill, res)
    interp = same & ((gfl & 0x10) == 0) & ((gfl & 1) != 0)
    ill = np.zeros(len(queries), bool)
    ill[interp] = cell_ill[qcells[interp]]
    qex, qev, qedge, qkmin = ol.trace(queries)
    if ill.any():
        both_v = (nv == 1) & (ev == 1)
        nerr = np.zeros((N, 3))
        nerr[both_v, 0] = np.abs(node6[both_v, 0:2] - ex[both_v, 0:2]).max(axis=1)
        nerr[both_v, 1] = np.abs(node6[both_v, 2:5] - ex[both_v, 2:5]).max(axis=1)
        nerr[both_v, 2] = np.abs(node6[both_v, 5] - ex[both_v, 5])
        cerr = corner_max(nerr, res)
        ci = qcells[ill]
        ep = np.abs(gout[ill, 0:2] - oout[ill, 0:2]).max(axis=1)
        ed = np.abs(gout[ill, 2:5] - oout[ill, 2:5]).max(axis=1)
        ei = np.abs(gout[ill, 5] - oout[ill, 5])
        assert np.all(ep <= POS_TOL + cerr[ci, 0]), f"{label}: ill-conditioned cell query position"
        assert np.all(ed <= DIR_TOL + cerr[ci, 1]), f"{label}: ill-conditioned cell query direction"
        assert np.all(ei <= I_TOL + cerr[ci, 2]), f"{label}: ill-conditioned cell query throughput"
    oval = np.where((ofl & 1) != 0, 1, 0).astype(np.uint8)
    oval[(ofl & 8) != 0] = 8
    keep = np.nonzero(same & ~ill)[0]
    q_st = compare_trace(gout[keep], gfl[keep], oout[keep], oval[keep], qedge[keep], qkmin[keep],
                         f"{label} query", cond=(ol, queries.subset(keep), (0, 0)))
    q_st["ill_cell_rays"] = int(ill.sum())
    frac = {"traced": float(((gfl & 0x10) != 0).mean()),
            "interpolated": float((((gfl & 0x10) == 0) & ((gfl & 1) != 0)).mean()),
            "mask_only": float((((gfl & 0x10) == 0) & ((gfl & 1) == 0)).mean())}
    # map error against the exact trace (reported, not bounded)
    v = ((gfl & 1) != 0) & (qev == 1) & ((gfl & 0x10) == 0)
    err = np.hypot(gout[v, 0] - qex[v, 0], gout[v, 1] - qex[v, 1])
    rep = {"class_mismatch": int(len(mism)), "node_pos_max": node_st["pos_max"],
           "query_pos_max": q_st["pos_max"], **frac,
           "map_err_rms_mm": float(np.sqrt((err ** 2).mean())) if v.any() else 0.0,
           "map_err_p99_mm": float(np.percentile(err, 99)) if v.any() else 0.0, **st}
    print(label, rep)
    return gmap, omap, rep


def test_singlet_map_full_size():
    p = w.singlet_lens()
    rays = w.singlet_rays()
    check_map(p, w.SINGLET_RHO, rays, rays, label="singlet 32^4x8")


@pytest.mark.slow
def test_eleven_map_full_size():
    p = w.eleven_surface_lens(oracle_accept)
    fit = w.eleven_fit_rays(p)
    q = w.eleven_rays(p)
    check_map(p, w.eleven_rho(p), fit, q, label="eleven 32^4x8")


def test_small_lattice_ragged_queries():
    p = w.singlet_lens()
    fit = w.singlet_rays(5000)
    q = w.entrance_rays(100003, 99, 13.0)      # some rays outside the box (r > 12)
    check_map(p, 12.0, fit, q, res=[5, 7, 4, 6, 3], label="small lattice")


def test_no_mask_ablation_overexposes():
    """Paper Fig. 6: without the valid/occluded mask every ray inside the box
    is taken as valid -- occluded rays reach the sensor (blurred image) and the
    summed throughput exceeds the true one."""
    p = w.singlet_lens()
    rays = w.singlet_rays()
    lo, hi = box(12.0)
    g = lt.Map.build(lt.Lens(p), 0, RES, lo, hi, fit=batch.DeviceRays(rays))
    o_mask, f_mask = gpu_query(g, rays, lt.QUERY_TABLE)
    o_nom, f_nom = gpu_query(g, rays, lt.QUERY_NO_MASK)
    ex, ev, _, _ = oracle.Lens(p).trace(rays)
    true_I = ex[ev == 1, 5].sum()
    assert abs(o_mask[:, 5].sum() - true_I) / true_I < 1e-3
    assert o_nom[:, 5].sum() > true_I
    assert ((f_nom & 1) != 0).mean() == 1.0
    # every occluded ray now produces an output; with the mask none does
    false_valid_nomask = (((f_nom & 1) != 0) & (ev != 1)).mean()
    false_valid_mask = (((f_mask & 1) != 0) & (ev != 1)).mean()
    assert false_valid_mask == 0.0 and false_valid_nomask > 0.25


def test_residual_limit_bounds_the_error_on_fit_rays():
    p = w.singlet_lens()
    rays = w.singlet_rays()
    lo, hi = box(12.0)
    lens = lt.Lens(p)
    g0 = lt.Map.build(lens, 0, RES, lo, hi, fit=batch.DeviceRays(rays))
    g1 = lt.Map.build(lens, 0, RES, lo, hi, fit=batch.DeviceRays(rays), max_residual_mm=1e-4)
    assert g1.stats()["cells_valid"] < g0.stats()["cells_valid"]
    out, fl = gpu_query(g1, rays)
    ex, ev, edge, kmin = oracle.Lens(p).trace(rays)
    v = ((fl & 1) != 0) & (ev == 1) & (kmin >= GRAZING_K) & (edge >= EDGE_EPS)
    err = np.hypot(out[v, 0] - ex[v, 0], out[v, 1] - ex[v, 1])
    assert err.max() <= 1e-4 + POS_TOL


def test_save_load_and_host_query_are_bitwise_equal():
    p = w.singlet_lens()
    rays = w.singlet_rays()
    lo, hi = box(12.0)
    g = lt.Map.build(lt.Lens(p), 0, [9, 9, 9, 9, 4], lo, hi, fit=batch.DeviceRays(rays))
    ref, rfl = gpu_query(g, rays)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "m.ltmap")
        g.save(path)
        g2 = lt.Map.load(path)
    out, fl = gpu_query(g2, rays)
    assert np.array_equal(out, ref) and np.array_equal(fl, rfl)
    assert g2.stats()["cells_valid"] == g.stats()["cells_valid"]
    h = batch.HostRays(rays)
    g.query_host(h.inp[:5], h.inp[5], h.out + [h.flags], len(rays))
    assert np.array_equal(np.stack([t.numpy() for t in h.out], 1), ref)
    assert np.array_equal(h.flags.numpy(), rfl)


@pytest.mark.parametrize("pin", [True, False, "mixed"])
def test_host_query_in_chunks_is_bitwise_equal(pin):
    # 600,001 rays: the device call runs the classify kernel and the queue
    # tracer over the whole batch, the host call four chunks (the last one
    # ragged) of the one-kernel query; pinned, pageable and mixed host arrays
    p = w.singlet_lens()
    rays = w.singlet_rays(600001)
    lo, hi = box(12.0)
    g = lt.Map.build(lt.Lens(p), 0, [9, 9, 9, 9, 4], lo, hi, fit=batch.DeviceRays(w.singlet_rays(20000)))
    ref, rfl = gpu_query(g, rays)
    h = batch.HostRays(rays, pin=(pin is True))
    if pin == "mixed":
        h.inp[:3] = [t.pin_memory() for t in h.inp[:3]]
    g.query_host(h.inp[:5], h.inp[5], h.out + [h.flags], len(rays))
    assert np.array_equal(np.stack([t.numpy() for t in h.out], 1), ref)
    assert np.array_equal(h.flags.numpy(), rfl)


def test_query_zero_rays():
    p = w.singlet_lens()
    lo, hi = box(12.0)
    g = lt.Map.build(lt.Lens(p), 0, [3, 3, 3, 3, 2], lo, hi)
    o = batch.DeviceOut(1)
    o.flags.fill_(9)
    d = batch.DeviceRays(w.singlet_rays(1))
    g.query(d.inp, d.lam, o.out, 0)
    torch.cuda.synchronize()
    assert int(o.flags[0]) == 9
