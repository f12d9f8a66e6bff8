"""Pins of the oracle's even aspheres (circularly symmetric surfaces, which
the paper's model admits, Sec. 4.1): the asphere route reduces to the
sphere's when kappa and the polynomial vanish; a Cartesian oval focuses
parallel light to a point; a polynomial surface is hit at its sag and
refracts about the normal of its derivative; reversibility holds."""
import dataclasses
import math
import types

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


def forced(presc, ks):
    """The same prescription with surfaces ks taken through the asphere route."""
    surfs = []
    for k, s in enumerate(presc.surfaces):
        d = dataclasses.asdict(s)
        if k + 1 in ks:
            d["force_asphere"] = True
        surfs.append(types.SimpleNamespace(**d))
    return dataclasses.replace(presc, surfaces=surfs)


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_zero_asphere_reduces_to_the_sphere(which):
    p = w.singlet_lens() if which == "singlet" else w.eleven_surface_lens(accept)
    rays = w.entrance_rays(3000, 5, 1.1 * p.surfaces[0].aperture_r)
    ref = oracle.Lens(p).trace(rays)
    got = oracle.Lens(forced(p, range(1, p.n_surfaces + 1))).trace(rays)
    assert np.array_equal(ref[1], got[1])
    v = ref[1] == 1
    assert np.abs(ref[0][v] - got[0][v]).max() < 1e-11
    for pid in sorted({1, min(3, p.n_surfaces * (p.n_surfaces - 1) // 2)}):
        path = oracle.path_ij(p.n_surfaces, pid)
        a = oracle.Lens(p).trace(rays, path)
        b = oracle.Lens(forced(p, range(1, p.n_surfaces + 1))).trace(rays, path)
        assert np.array_equal(a[1], b[1])
        v = a[1] == 1
        assert np.abs(a[0][v] - b[0][v]).max() < 1e-9


def cartesian_oval(n=1.6, R1=40.0, t=6.0, a=12.0):
    """Air -> glass ellipsoid kappa = -1/n^2 (focuses parallel light to its far
    focus F = n R / (n - 1) behind the vertex), then a sphere centred on F
    (rays cross it along radii), image plane on F."""
    F = n * R1 / (n - 1.0)
    g = w.Glass(kind=w.GLASS_CAUCHY, A=n, B=0.0)
    s1 = w.Surface(1.0 / R1, t, a, 0, conic=-1.0 / n ** 2)
    s2 = w.Surface(1.0 / (F - t), 0.0, a, -1)
    return w.Prescription(surfaces=[s1, s2], glasses=[g], entrance_gap=1.0, stop_after=0, stop_r=0.0,
                          image_mode=w.IMAGE_ABS, image_z=1.0 + F), F


def test_cartesian_oval_focuses_parallel_light_to_a_point():
    p, F = cartesian_oval()
    ol = oracle.Lens(p)
    rng = np.random.default_rng(3)
    for _ in range(200):
        r, phi = 11.0 * math.sqrt(rng.uniform()), rng.uniform(0, 2 * math.pi)
        v, o, _, _ = ol.trace_one(r * math.cos(phi), r * math.sin(phi), 0.0, 0.0, 1.0, 550.0)
        assert v == 1
        assert abs(o[0]) < 1e-10 and abs(o[1]) < 1e-10
    # the same surface as a sphere (kappa = 0) does not: spherical aberration
    q = dataclasses.replace(p, surfaces=[dataclasses.replace(p.surfaces[0], conic=0.0), p.surfaces[1]])
    v, o, _, _ = oracle.Lens(q).trace_one(10.0, 0.0, 0.0, 0.0, 1.0, 550.0)
    assert v == 1 and abs(o[0]) > 1e-2


def test_polynomial_surface_hit_and_normal():
    A4, A6 = 2e-4, -3e-7
    n = 1.5
    g = w.Glass(kind=w.GLASS_CAUCHY, A=n, B=0.0)
    s1 = w.Surface(0.0, 4.0, 10.0, 0, asph=(A4, A6, 0.0, 0.0))
    s2 = w.Surface(0.0, 0.0, 10.0, -1)
    p = w.Prescription(surfaces=[s1, s2], glasses=[g], entrance_gap=2.0, stop_r=0.0,
                       image_mode=w.IMAGE_ABS, image_z=30.0)
    ol = oracle.Lens(p)
    h = 7.0
    v, o, st = ol.trace_states(h, 0.0, 0.0, 0.0, 1.0, 550.0)
    assert v == 1
    hit = st[0]
    sag = A4 * h ** 4 + A6 * h ** 6
    assert abs(hit[0] - h) < 1e-12 and abs(hit[2] - (2.0 + sag)) < 1e-12
    # refraction about the normal facing the ray, (z'(h), 0, -1) / |.|,
    # z'(h) = 4 A4 h^3 + 6 A6 h^5 (vector Snell's law written out by hand)
    slope = 4 * A4 * h ** 3 + 6 * A6 * h ** 5
    nrm = np.array([slope, 0.0, -1.0]) / math.hypot(slope, 1.0)
    d = np.array([0.0, 0.0, 1.0])
    ci = -float(nrm @ d)
    eta = 1.0 / n
    k = 1.0 - eta * eta * (1.0 - ci * ci)
    t = eta * d + (eta * ci - math.sqrt(k)) * nrm
    assert np.allclose(hit[3:6], t / np.linalg.norm(t), atol=1e-13)


def test_reversibility_with_aspheres():
    p = w.eleven_surface_lens(accept)
    surfs = list(p.surfaces)
    surfs[1] = dataclasses.replace(surfs[1], conic=-0.6, asph=(3e-6, -1e-9, 0.0, 0.0))
    surfs[8] = dataclasses.replace(surfs[8], conic=0.4, asph=(-2e-6, 0.0, 0.0, 0.0))
    p = dataclasses.replace(p, surfaces=surfs)
    fwd = oracle.Lens(p)
    back = oracle.Lens(R.reverse_prescription(p, fwd.z_image(), 0.0, w.IMAGE_ABS))
    rays = w.entrance_rays(300, 8, 0.8 * p.surfaces[0].aperture_r)
    checked = 0
    for r in range(len(rays)):
        a = [float(x[r]) for x in rays.arrays()]
        v, o, edge, kmin = fwd.trace_one(*a)
        if v != 1 or edge < 1e-6 or kmin < 1e-2:
            continue
        vb, ob, _, _ = back.trace_one(o[0], o[1], -o[2], -o[3], o[4], a[5])
        assert vb == 1
        assert abs(ob[0] - a[0]) < 1e-8 and abs(ob[1] - a[1]) < 1e-8
        assert abs(ob[5] - o[5]) < 1e-12
        checked += 1
    assert checked > 50
