"""GPU parity of the FP32 tracer (lt_trace) against the FP64 oracle, through
the C ABI: the 2-surface singlet (all 65,536 rays, transmission and ghost),
the seeded 11-surface lens at its full 4,194,304-ray size, every ghost path
of that lens, ragged sizes, bad inputs and the host-buffer entry point."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import compare_trace

pytestmark = pytest.mark.gpu


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def eleven():
    return w.eleven_surface_lens(oracle_accept)


def run_gpu(lens, rays, path_id, stream=None):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    lt.trace(lens, d.inp, d.lam, path_id, o.out, len(rays), stream)
    torch.cuda.synchronize()
    return o.numpy()


@pytest.mark.parametrize("path_id", [0, 1])
def test_singlet_all_rays(path_id):
    p = w.singlet_lens()
    rays = w.singlet_rays()
    out, flags = run_gpu(lt.Lens(p), rays, path_id)
    ol = oracle.Lens(p)
    path = oracle.path_ij(2, path_id)
    ex, ev, edge, kmin = ol.trace(rays, path)
    st = compare_trace(out, flags, ex, ev, edge, kmin, f"singlet path {path_id}",
                       cond=(ol, rays, path))
    assert st["valid_gpu"] > 1000


def test_eleven_full_size_transmission(eleven):
    rays = w.eleven_rays(eleven)          # 4,194,304 rays
    out, flags = run_gpu(lt.Lens(eleven), rays, 0)
    ol = oracle.Lens(eleven)
    ex, ev, edge, kmin = ol.trace(rays)
    st = compare_trace(out, flags, ex, ev, edge, kmin, "eleven transmission",
                       cond=(ol, rays, (0, 0)))
    assert st["valid_gpu"] > 100000


def test_eleven_every_ghost_path(eleven):
    lens = lt.Lens(eleven)
    ol = oracle.Lens(eleven)
    rays = w.eleven_rays(eleven, 20000)
    S = eleven.n_surfaces
    worst = {"pos_max": 0.0, "dir_max": 0.0, "I_max": 0.0}
    for pid in range(1, lens.n_paths):
        out, flags = run_gpu(lens, rays, pid)
        path = oracle.path_ij(S, pid)
        ex, ev, edge, kmin = ol.trace(rays, path)
        st = compare_trace(out, flags, ex, ev, edge, kmin, f"eleven ghost {pid}",
                           cond=(ol, rays, path))
        for k in worst:
            worst[k] = max(worst[k], st[k])
    print("ghost worst", worst)


@pytest.mark.parametrize("n", [1, 31, 255, 257, 4097, 100003])
def test_ragged_sizes(n):
    p = w.singlet_lens()
    rays = w.singlet_rays(n)
    out, flags = run_gpu(lt.Lens(p), rays, 0)
    ol = oracle.Lens(p)
    ex, ev, edge, kmin = ol.trace(rays)
    compare_trace(out, flags, ex, ev, edge, kmin, f"ragged {n}", cond=(ol, rays, (0, 0)))


def test_zero_rays_is_a_noop():
    lens = lt.Lens(w.singlet_lens())
    o = batch.DeviceOut(1)
    o.flags.fill_(77)
    rays = w.singlet_rays(1)
    d = batch.DeviceRays(rays)
    lt.trace(lens, d.inp, d.lam, 0, o.out, 0)
    torch.cuda.synchronize()
    assert int(o.flags[0]) == 77


def test_bad_inputs_are_flagged():
    p = w.singlet_lens()
    rays = w.singlet_rays(64)
    rays.x[0] = np.nan
    rays.dz[1] = -0.5
    rays.lam[2] = 0.0
    rays.dy[3] = np.inf
    out, flags = run_gpu(lt.Lens(p), rays, 0)
    ol = oracle.Lens(p)
    ex, ev, edge, kmin = ol.trace(rays)
    compare_trace(out, flags, ex, ev, edge, kmin, "bad inputs", cond=(ol, rays, (0, 0)))
    assert np.all(flags[:4] == lt.FLAG_BAD_INPUT)


@pytest.mark.parametrize("pin", [True, False])
def test_host_entry_point_is_bitwise_equal(eleven, pin):
    # pinned and pageable host arrays; 300,001 rays run as four chunks of the
    # three-stream pipeline, the last one ragged
    lens = lt.Lens(eleven)
    rays = w.eleven_rays(eleven, 300001)
    out_d, flags_d = run_gpu(lens, rays, 3)
    h = batch.HostRays(rays, pin=pin)
    lt.trace_host(lens, h.inp[:5], h.inp[5], 3, h.out + [h.flags], len(rays))
    out_h = np.stack([t.numpy() for t in h.out], axis=1)
    assert np.array_equal(out_h, out_d)
    assert np.array_equal(h.flags.numpy(), flags_d)


def test_side_stream(eleven):
    lens = lt.Lens(eleven)
    rays = w.eleven_rays(eleven, 50000)
    ref, fref = run_gpu(lens, rays, 0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out, flags = run_gpu(lens, rays, 0, stream=s)
    assert np.array_equal(out, ref) and np.array_equal(flags, fref)


def test_near_edge_flag_band_is_tight():
    """Rays placed at known distances from the singlet's stop edge (r = 10 mm
    at z = 0): the flag marks exactly the ones within 1e-6 mm (up to FP32
    resolution of r^2 at r = 10)."""
    p = w.singlet_lens()
    offs = np.array([-1e-3, -1e-5, -3e-7, 0.0, 3e-7, 1e-5, 1e-3])
    n = len(offs)
    f = np.float32
    rays = w.Rays(x=(10.0 + offs).astype(f), y=np.zeros(n, f), dx=np.zeros(n, f),
                  dy=np.zeros(n, f), dz=np.ones(n, f), lam=np.full(n, 550.0, f))
    out, flags = run_gpu(lt.Lens(p), rays, 0)
    near = (flags & lt.FLAG_NEAR_EDGE) != 0
    assert list(near) == [False, False, True, True, True, False, False]
    assert list((flags & 1) != 0)[:2] == [True, True]
    assert list((flags & 1) != 0)[-2:] == [False, False]


@pytest.mark.parametrize("lens_kind", ["singlet", "eleven"])
def test_profiler_counts_every_interaction(lens_kind, eleven):
    """The profiler's work count (ray-surface interactions evaluated, the image
    plane counting as one) is exact: near-axis rays that all pass the lens
    count K + 1 each, and a count over the whole batch equals the counts of
    its two halves traced separately."""
    p = w.singlet_lens() if lens_kind == "singlet" else eleven
    lens = lt.Lens(p)
    S = p.n_surfaces
    rays = w.entrance_rays(200003, 5, 1.0, half_angle_deg=0.5)
    ol = oracle.Lens(p)
    _, ev, _, _ = ol.trace(rays, oracle.path_ij(S, 0))
    assert np.all(ev == 1)
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    n = len(rays)
    lt.profile_enable(True)
    try:
        lt.profile_read(reset=True)
        lt.trace(lens, d.inp, d.lam, 0, o.out, n)
        whole = lt.profile_read(reset=True)["trace_kernel"]
        assert whole[0] == 1 and whole[2] == (S + 1) * n
        # a ghost path, where rays die at many depths: whole batch = sum of halves
        lt.trace(lens, d.inp, d.lam, 1, o.out, n)
        g = lt.profile_read(reset=True)["trace_kernel"][2]
        h = (n // 2) & ~63          # keeps the second half's arrays 16-byte aligned
        lt.trace(lens, [t[:h] for t in d.inp], d.lam[:h], 1, o.out, h)
        lt.trace(lens, [t[h:] for t in d.inp], d.lam[h:], 1, [t[h:] for t in o.out], n - h)
        halves = lt.profile_read(reset=True)["trace_kernel"]
        assert halves[0] == 2 and halves[2] == g and g > 0
    finally:
        lt.profile_enable(False)
