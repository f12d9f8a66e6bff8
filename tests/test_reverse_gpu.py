"""Backward path tracing (Sec. 3, Eq. 9) through lt_reverse_lens: the
library's reversed lens traced on the GPU against the oracle's own reversal
of the prescription, element by element; a forward trace followed by the
backward trace of its reversed exit rays; and the backward (full
transmission) map of the paper's depth-of-field rendering -- a table map of
the reversed lens -- against the oracle's map of the same reversed lens."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import reverse as R
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import EDGE_EPS, GRAZING_K, compare_trace
from test_map_gpu import check_map

pytestmark = pytest.mark.gpu


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module", params=["singlet", "eleven"])
def lens(request):
    return w.singlet_lens() if request.param == "singlet" else w.eleven_surface_lens(oracle_accept)


def sensor_rays(n, seed, rho, half_angle_deg=15.0):
    """Rays leaving the sensor towards the lens, in the reversed lens's frame."""
    return w.entrance_rays(n, seed, rho, half_angle_deg)


def run(lens_h, rays, path=0):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    lt.trace(lens_h, d.inp, d.lam, path, o.out, len(rays))
    torch.cuda.synchronize()
    return o.numpy()


def test_backward_trace_matches_oracle(lens):
    fwd = lt.Lens(lens)
    zi = fwd.paraxial(w.LAMBDA_D_NM)[2]
    for sensor_z, out_z in ((zi, 0.0), (zi + 0.6, -2.0)):   # in focus, and refocused
        back = fwd.reversed(sensor_z, out_z)
        ol = oracle.Lens(R.reverse_prescription(lens, sensor_z, out_z, w.IMAGE_ABS))
        rays = sensor_rays(200000, 31, 9.0)
        out, flags = run(back, rays)
        ex, ev, edge, kmin = ol.trace(rays)
        st = compare_trace(out, flags, ex, ev, edge, kmin, f"backward sensor_z={sensor_z:.3f}",
                           cond=(ol, rays, (0, 0)))
        assert st["valid_gpu"] > 5000


def test_forward_then_backward_returns_to_the_entrance(lens):
    fwd = lt.Lens(lens)
    zi = fwd.paraxial(w.LAMBDA_D_NM)[2]
    back = fwd.reversed(zi, 0.0)
    rays = w.entrance_rays(100000, 32, 0.8 * lens.surfaces[0].aperture_r)
    out, flags = run(fwd, rays)
    ok = ((flags & lt.FLAG_VALID) != 0) & ((flags & (lt.FLAG_NEAR_EDGE | lt.FLAG_NEAR_TIR | lt.FLAG_GRAZING)) == 0)
    rev = w.Rays(out[ok, 0].copy(), out[ok, 1].copy(), -out[ok, 2], -out[ok, 3], out[ok, 4].copy(),
                 rays.lam[ok].copy())
    bout, bflags = run(back, rev)
    v = (bflags & lt.FLAG_VALID) != 0
    assert v.mean() > 0.999
    src = rays.subset(np.nonzero(ok)[0])
    n = np.sqrt(src.dx.astype(np.float64) ** 2 + src.dy ** 2 + src.dz ** 2)
    assert np.abs(bout[v, 0] - src.x[v]).max() < 2e-3
    assert np.abs(bout[v, 1] - src.y[v]).max() < 2e-3
    assert np.abs(bout[v, 2] + src.dx[v] / n[v]).max() < 1e-5
    assert np.abs(bout[v, 4] - src.dz[v] / n[v]).max() < 1e-5
    assert np.abs(bout[v, 5] - out[ok, 5][v]).max() < 1e-5     # Fresnel transmission is reciprocal


def test_backward_map_matches_oracle_map():
    p = w.singlet_lens()
    fwd = lt.Lens(p)
    zi = fwd.paraxial(w.LAMBDA_D_NM)[2]
    back = fwd.reversed(zi, 0.0)
    ol = oracle.Lens(R.reverse_prescription(p, zi, 0.0, w.IMAGE_ABS))
    smax = math.tan(math.radians(15.0))
    fit = sensor_rays(40000, 33, 9.0)
    q = sensor_rays(60001, 34, 9.2)            # a few fall outside the lattice box
    _, _, rep = check_map(p, 9.0, fit, q, res=[12, 12, 12, 12, 4], label="backward map",
                          lens=back, ol=ol, smax=smax)
    assert rep["interpolated"] > 0.1
