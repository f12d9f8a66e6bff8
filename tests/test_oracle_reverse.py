"""Pins of the oracle's reversed lens (backward path tracing, Sec. 3, Eq. 9):
reversibility of the FP64 trace through the mirrored prescription, the
focal length seen from the other side, and the stop's place."""
import numpy as np
import pytest

import oracle
from oracle import reverse as R
from paper_2605_04017_gb300 import workloads as w


def accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module", params=["singlet", "eleven"])
def lens(request):
    return w.singlet_lens() if request.param == "singlet" else w.eleven_surface_lens(accept)


def reversed_oracle(p, sensor_z, out_z):
    return oracle.Lens(R.reverse_prescription(p, sensor_z, out_z, w.IMAGE_ABS))


def test_backward_trace_returns_to_the_entrance_ray(lens):
    fwd = oracle.Lens(lens)
    zi = fwd.z_image()
    back = reversed_oracle(lens, zi, 0.0)
    rays = w.entrance_rays(400, 99, 0.8 * lens.surfaces[0].aperture_r)
    checked = 0
    for r in range(len(rays)):
        a = [float(v[r]) for v in rays.arrays()]
        v, o, edge, kmin = fwd.trace_one(*a)
        if v != 1 or edge < 1e-6 or kmin < 1e-2:
            continue
        vb, ob, _, _ = back.trace_one(o[0], o[1], -o[2], -o[3], o[4], a[5])
        assert vb == 1
        assert abs(ob[0] - a[0]) < 1e-9 and abs(ob[1] - a[1]) < 1e-9
        n = np.sqrt(a[2] ** 2 + a[3] ** 2 + a[4] ** 2)
        assert np.allclose(ob[2:5], [-a[2] / n, -a[3] / n, a[4] / n], atol=1e-12)
        assert abs(ob[5] - o[5]) < 1e-12            # Fresnel transmission is reciprocal
        checked += 1
    assert checked > 100


def test_focal_length_is_the_same_from_both_sides(lens):
    fwd = oracle.Lens(lens)
    back = reversed_oracle(lens, fwd.z_image(), 0.0)
    for lam in (400.0, 587.6, 760.0):
        assert back.paraxial(lam)[0] == pytest.approx(fwd.paraxial(lam)[0], rel=1e-12)


def test_stop_keeps_its_plane():
    p = w.eleven_surface_lens(accept)
    fwd = oracle.Lens(p)
    sensor_z, out_z = fwd.z_image() + 0.7, -3.0
    back = reversed_oracle(p, sensor_z, out_z)
    assert back.z_stop() == pytest.approx(sensor_z - fwd.z_stop(), abs=1e-12)
    assert back.z_image() == pytest.approx(sensor_z - out_z, abs=1e-12)
    # the symmetric singlet: its stop sits on the front vertex, which becomes the back one
    s = w.singlet_lens()
    fs = oracle.Lens(s)
    bs = reversed_oracle(s, fs.z_image(), 0.0)
    assert bs.z_stop() == pytest.approx(fs.z_image(), abs=1e-12)
