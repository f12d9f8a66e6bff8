"""Even aspheres on the GPU (the tracer's general instantiation): an
11-surface lens with three aspheric surfaces traced against the oracle,
element by element, on the main path and ghost paths; a Cartesian oval
focusing parallel light to a point; and a table map of the aspheric lens
against the oracle's map."""
import dataclasses
import math

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


@pytest.fixture(scope="module")
def aspheric():
    p = w.eleven_surface_lens(oracle_accept)
    s = list(p.surfaces)
    s[1] = dataclasses.replace(s[1], conic=-0.6, asph=(3e-6, -1e-9, 0.0, 0.0))
    s[4] = dataclasses.replace(s[4], conic=0.0, asph=(0.0, 2e-9, -1e-12, 0.0))
    s[8] = dataclasses.replace(s[8], conic=0.4, asph=(-2e-6, 0.0, 0.0, 1e-15))
    return dataclasses.replace(p, surfaces=s)


def run(lens, rays, path_id=0):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    lt.trace(lens, d.inp, d.lam, path_id, o.out, len(rays))
    torch.cuda.synchronize()
    return o.numpy()


def test_aspheric_lens_matches_oracle(aspheric):
    lens, ol = lt.Lens(aspheric), oracle.Lens(aspheric)
    rays = w.eleven_rays(aspheric, 200000)
    out, flags = run(lens, rays)
    ex, ev, edge, kmin = ol.trace(rays)
    st = compare_trace(out, flags, ex, ev, edge, kmin, "aspheric main", cond=(ol, rays, (0, 0)))
    assert st["valid_gpu"] > 20000
    # the aspheres matter: the spherical lens gives other exits
    sph = lt.Lens(w.eleven_surface_lens(oracle_accept))
    o2, f2 = run(sph, rays)
    both = ((flags & 1) != 0) & ((f2 & 1) != 0)
    assert np.abs(out[both, 0] - o2[both, 0]).max() > 1e-2
    S = aspheric.n_surfaces
    small = w.eleven_rays(aspheric, 20000)
    for pid in (1, 12, 40, 55):
        path = oracle.path_ij(S, pid)
        o, f = run(lens, small, pid)
        gx, gv, ge, gk = ol.trace(small, path)
        compare_trace(o, f, gx, gv, ge, gk, f"aspheric ghost {pid}", cond=(ol, small, path))


def test_cartesian_oval_focuses_on_the_gpu():
    n, R1, t, a = 1.6, 40.0, 6.0, 12.0
    F = n * R1 / (n - 1.0)
    g = w.Glass(kind=w.GLASS_CAUCHY, A=n, B=0.0)
    p = w.Prescription(surfaces=[w.Surface(1.0 / R1, t, a, 0, conic=-1.0 / n ** 2), w.Surface(1.0 / (F - t), 0.0, a, -1)],
                       glasses=[g], entrance_gap=1.0, stop_r=0.0, image_mode=w.IMAGE_ABS, image_z=1.0 + F)
    N = 50000
    rng = np.random.default_rng(4)
    r = 11.0 * np.sqrt(rng.uniform(size=N))
    phi = rng.uniform(0, 2 * math.pi, N)
    rays = w.Rays((r * np.cos(phi)).astype(np.float32), (r * np.sin(phi)).astype(np.float32),
                  np.zeros(N, np.float32), np.zeros(N, np.float32), np.ones(N, np.float32),
                  np.full(N, 550.0, np.float32))
    out, flags = run(lt.Lens(p), rays)
    assert ((flags & 1) != 0).all()
    assert np.abs(out[:, 0]).max() < 1e-4 and np.abs(out[:, 1]).max() < 1e-4


def test_aspheric_map_matches_oracle_map(aspheric):
    rho = w.eleven_rho(aspheric)
    fit = w.eleven_rays(aspheric, 60000)
    q = w.entrance_rays(50001, 77, rho)
    _, _, rep = check_map(aspheric, rho, fit, q, res=[10, 10, 10, 10, 4], label="aspheric map")
    assert rep["traced"] > 0.0 and rep["interpolated"] > 0.0
