"""GPU parity on lens variants the seeded workloads do not cover, through the
C ABI against the oracle:
  - a lens mixing Sellmeier and Cauchy glass (the general-dispersion tracer
    path, which every all-Cauchy lens skips), traced, mapped, traced along
    every flare path in one launch, and served by the fused request kernel;
  - the maximum-size lens (32 surfaces) including all 497 of its paths in
    one lt_trace_paths launch;
  - a stop after the last surface, an absolute image plane, and plane
    surfaces (a plano-convex element and a plane-parallel plate).
Glass coefficients here are synthetic."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import compare_trace
from test_map_gpu import check_map

pytestmark = pytest.mark.gpu


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


def sellmeier_mix():
    """The 11-surface lens with every other glass replaced by a synthetic
    3-term Sellmeier glass of about the same index at 587.6 nm."""
    el = w.eleven_surface_lens(oracle_accept)
    gl = []
    for k, g in enumerate(el.glasses):
        if k % 2 == 0:
            n0 = g.A + g.B / 0.5876 ** 2
            b1 = (n0 ** 2 - 1) * (1 - 0.012 / 0.5876 ** 2)
            gl.append(w.Glass(kind=w.GLASS_SELLMEIER, B3=(b1, 0.05, 0.8), C3=(0.012, 0.04, 95.0)))
        else:
            gl.append(g)
    return dataclasses.replace(el, glasses=gl)


def run_gpu(lens, rays, path_id):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    lt.trace(lens, d.inp, d.lam, path_id, o.out, len(rays))
    torch.cuda.synchronize()
    return o.numpy()


def check_paths(presc, rays, pids, label):
    lens = lt.Lens(presc)
    ol = oracle.Lens(presc)
    for pid in pids:
        out, flags = run_gpu(lens, rays, pid)
        path = oracle.path_ij(presc.n_surfaces, pid)
        ex, ev, edge, kmin = ol.trace(rays, path)
        compare_trace(out, flags, ex, ev, edge, kmin, f"{label} path {pid}", cond=(ol, rays, path))


@pytest.fixture(scope="module")
def mix():
    return sellmeier_mix()


def test_sellmeier_mix_trace(mix):
    rays = w.entrance_rays(20000, 31, w.eleven_rho(mix))
    check_paths(mix, rays, [0, 1, 7, 30, 55], "sellmeier mix")


def test_sellmeier_mix_map(mix):
    rho = w.eleven_rho(mix)
    fit = w.entrance_rays(200000, 32, rho)
    queries = w.entrance_rays(50000, 33, rho)
    check_map(mix, rho, fit, queries, res=[12, 12, 12, 12, 4], label="sellmeier mix map")


def test_sellmeier_mix_flare_launch_and_server(mix):
    lens = lt.Lens(mix)
    ol = oracle.Lens(mix)
    n = 700
    rays = w.entrance_rays(n, 34, w.eleven_rho(mix))
    P = lens.n_paths
    lam = np.stack([w.redraw_wavelengths(n, 500 + p) for p in range(P)])
    d = batch.DeviceRays(rays)
    dl = torch.from_numpy(lam.reshape(-1)).cuda()
    po = batch.PathsOut(P, n)
    lt.trace_paths(lens, d.inp, dl, n, list(range(P)), po, n)
    torch.cuda.synchronize()
    for p in range(P):
        idx, out, flags = po.path(p)
        full = np.zeros((n, 6), np.float32)
        fl = np.zeros(n, np.uint8)
        full[idx] = out
        fl[idx] = flags
        rp = dataclasses.replace(rays, lam=lam[p])
        path = oracle.path_ij(mix.n_surfaces, p)
        ex, ev, edge, kmin = ol.trace(rp, path)
        compare_trace(full, fl, ex, ev, edge, kmin, f"mix flare {p}", cond=(ol, rp, path))
    # the server's fused kernel (general-dispersion variant) equals lt_trace bit for bit
    srv = lt.Server()
    outs = []
    for pid in (0, 3, 17):
        o = batch.DeviceOut(n)
        outs.append((pid, o, srv.submit_trace(lens, d.inp, d.lam, pid, o.out, n)))
    for pid, o, t in outs:
        srv.wait(t)
        ref = run_gpu(lens, rays, pid)
        got = o.numpy()
        assert np.array_equal(got[0].view(np.uint32), ref[0].view(np.uint32)) and np.array_equal(got[1], ref[1])
    srv.close()


@pytest.fixture(scope="module")
def s32():
    return w.generate_lens(w.SEED_BASE + 77, 32, oracle_accept)


def test_32_surfaces_trace(s32):
    rays = w.entrance_rays(8000, 35, 1.2 * s32.surfaces[0].aperture_r)
    S = 32
    pids = [0, lt.path_id(S, 1, 2), lt.path_id(S, 1, 32), lt.path_id(S, 16, 17), lt.path_id(S, 31, 32)]
    check_paths(s32, rays, pids, "S=32")


def test_32_surfaces_every_path_one_launch(s32):
    lens = lt.Lens(s32)
    ol = oracle.Lens(s32)
    n = 300
    rays = w.entrance_rays(n, 36, 1.2 * s32.surfaces[0].aperture_r)
    P = lens.n_paths
    assert P == 1 + 32 * 31 // 2
    d = batch.DeviceRays(rays)
    po = batch.PathsOut(P, n)
    lt.trace_paths(lens, d.inp, d.lam, 0, list(range(P)), po, n)
    torch.cuda.synchronize()
    counts = po.counts()
    for p in range(P):
        idx, out, flags = po.path(p)
        full = np.zeros((n, 6), np.float32)
        fl = np.zeros(n, np.uint8)
        full[idx] = out
        fl[idx] = flags
        path = oracle.path_ij(32, p)
        ex, ev, edge, kmin = ol.trace(rays, path)
        compare_trace(full, fl, ex, ev, edge, kmin, f"S=32 launch {p}", cond=(ol, rays, path))
    print("S=32 valid rays over all paths", int(counts.sum()))


def test_stop_after_last_surface():
    p = dataclasses.replace(w.singlet_lens(), stop_after=2, stop_offset=3.0, stop_r=9.0)
    check_paths(p, w.singlet_rays(30000), [0, 1], "stop after last")


def test_absolute_image_plane():
    p = dataclasses.replace(w.singlet_lens(), image_mode=w.IMAGE_ABS, image_z=60.0)
    check_paths(p, w.singlet_rays(30000), [0, 1], "absolute image")


def test_plane_surfaces():
    p = w.Prescription(surfaces=[w.Surface(1 / 40.0, 4.0, 10.0, 0), w.Surface(0.0, 3.0, 10.0, -1),
                                 w.Surface(0.0, 2.0, 10.0, 1), w.Surface(0.0, 0.0, 10.0, -1)],
                       glasses=[w.Glass(kind=w.GLASS_CAUCHY, A=1.5, B=0.004),
                                w.Glass(kind=w.GLASS_CAUCHY, A=1.6, B=0.008)],
                       entrance_gap=1.0, stop_after=0, stop_offset=0.5, stop_r=9.5)
    check_paths(p, w.entrance_rays(30000, 37, 11.0), list(range(1 + 4 * 3 // 2)), "plane surfaces")
