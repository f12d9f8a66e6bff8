"""CPU checks that the seeded input generators produce the workloads the
benchmark and the parity tests claim: the singlet of the first workload
exactly, generated lenses within their parameter ranges and glass pattern,
and entrance rays with the stated distributions (uniform on the disk,
direction angles uniform within +-10 degrees, wavelengths uniform on
380-780 nm)."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04017_gb300 import workloads as w


def accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


def test_singlet_is_the_stated_prescription():
    p = w.singlet_lens()
    s1, s2 = p.surfaces
    assert (1 / s1.curvature, 1 / s2.curvature) == pytest.approx((50.0, -50.0))
    assert s1.thickness == 5.0 and s1.aperture_r == s2.aperture_r == 10.0
    assert s1.glass_after == 0 and s2.glass_after == -1
    g = p.glasses[0]
    assert g.kind == w.GLASS_CAUCHY and (g.A, g.B) == (1.5046, 0.00420)
    assert p.stop_after == 0 and p.stop_r == 10.0 and p.entrance_gap == 0.0
    assert p.image_mode == w.IMAGE_PARAXIAL


def test_eleven_surface_lens_follows_the_recipe():
    p = w.eleven_surface_lens(accept)
    assert p.n_surfaces == 11
    glass = [s.glass_after >= 0 for s in p.surfaces]
    assert glass == [True, False, True, False, True, False, True, True, False, True, False]
    assert p.stop_after == 6                       # the stop between surfaces 6 and 7, in air
    for s in p.surfaces:
        assert 20.0 <= abs(1.0 / s.curvature) <= 200.0
        assert 8.0 <= s.aperture_r <= 15.0
    for s in p.surfaces[:-1]:
        assert 1.0 <= s.thickness <= 8.0
    assert len(p.glasses) == 6                    # one per glass medium, cemented pair included
    for g in p.glasses:
        assert g.kind == w.GLASS_CAUCHY and 1.48 <= g.A <= 1.75 and 0.003 <= g.B <= 0.012
    assert p.stop_r == min(p.surfaces[5].aperture_r, p.surfaces[6].aperture_r)
    assert p.stop_offset == pytest.approx(0.5 * p.surfaces[5].thickness)
    assert accept(p)
    # consecutive surfaces keep 0.5 mm of clearance over the smaller aperture
    z = p.vertex_z()
    for k in range(10):
        a = min(p.surfaces[k].aperture_r, p.surfaces[k + 1].aperture_r)
        r = np.linspace(0.0, a, 65)
        sag = lambda c: c * r * r / (1.0 + np.sqrt(np.maximum(0.0, 1.0 - c * c * r * r)))  # noqa: E731
        gap = z[k + 1] + sag(p.surfaces[k + 1].curvature) - z[k] - sag(p.surfaces[k].curvature)
        assert gap.min() >= 0.5 - 1e-9


def test_serving_lenses_span_4_to_22_surfaces():
    lenses = w.serving_lenses(accept, 8)
    assert len(lenses) == 8
    assert all(4 <= p.n_surfaces <= 22 for p in lenses)
    assert all(accept(p) for p in lenses)


def test_entrance_rays_have_the_stated_distributions():
    n = 200000
    rho = 12.0
    r = w.entrance_rays(n, 123, rho)
    x, y, dx, dy, dz, lam = [a.astype(np.float64) for a in r.arrays()]
    rr = np.hypot(x, y)
    assert rr.max() <= rho * (1 + 1e-6)
    # uniform on the disk: r^2 / rho^2 is uniform on [0, 1]
    u = np.sort(rr ** 2 / rho ** 2)
    assert np.abs(u - (np.arange(n) + 0.5) / n).max() < 0.01
    assert np.abs(np.arctan2(y, x).mean()) < 0.02
    # unit directions, theta_x = atan(dx / dz) uniform within +-10 degrees
    assert np.abs(dx * dx + dy * dy + dz * dz - 1).max() < 1e-6
    tx = np.degrees(np.arctan2(dx, dz))
    ty = np.degrees(np.arctan2(dy, dz))
    assert tx.min() >= -10.0 - 1e-4 and tx.max() <= 10.0 + 1e-4
    assert np.abs(np.sort(tx) - (-10 + 20 * (np.arange(n) + 0.5) / n)).max() < 0.2
    assert abs(np.corrcoef(tx, ty)[0, 1]) < 0.01
    assert lam.min() >= 380.0 and lam.max() <= 780.0
    assert np.abs(np.sort(lam) - (380 + 400 * (np.arange(n) + 0.5) / n)).max() < 4.0
    # seeded: the same seed gives the same arrays, another seed others
    r2, r3 = w.entrance_rays(1000, 123, rho), w.entrance_rays(1000, 123, rho)
    assert all(np.array_equal(a, b) for a, b in zip(r2.arrays(), r3.arrays()))
    assert not np.array_equal(r2.x, w.entrance_rays(1000, 124, rho).x)


def test_flare_wavelengths_are_redrawn_per_path():
    a, b = w.flare_wavelengths(0, 4096), w.flare_wavelengths(1, 4096)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, w.flare_wavelengths(0, 4096))
    assert a.min() >= 380.0 and a.max() <= 780.0
