"""Pins for the oracle's FP64 tracer: each check compares it against something
other than itself -- a closed form, a physical invariant, a hand-enumerated
case, a catalogue value or a number printed in the paper.

A plausible slip anywhere in the tracer (a dropped Fresnel term, a wrong
normal sign, a swapped n1/n2 on a backward segment, a wrong reflection
order in a ghost path, a stop tested in the wrong gap) fails at least one.
"""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2605_04017_gb300 import workloads as w

LD = w.LAMBDA_D_NM


def singlet():
    return oracle.Lens(w.singlet_lens())


def oracle_accept(p):
    try:
        L = oracle.Lens(p)
        efl, bfd = L.paraxial(w.LAMBDA_D_NM)
        return efl > 0 and bfd > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def eleven():
    return w.eleven_surface_lens(oracle_accept)


def cauchy_n(lam_nm, A=1.5046, B=0.00420):
    return A + B / (lam_nm * 1e-3) ** 2


# ---------------------------------------------------------------- paraxial

@pytest.mark.parametrize("lam", [380.0, LD, 780.0])
def test_paraxial_singlet_matches_thick_lens_formula(lam):
    """Thick-lens lensmaker formula (closed form, not a matrix product)."""
    n = cauchy_n(lam)
    R1, R2, t = 50.0, -50.0, 5.0
    inv_f = (n - 1) * (1 / R1 - 1 / R2 + (n - 1) * t / (n * R1 * R2))
    f = 1 / inv_f
    bfd = f * (1 - (n - 1) * t / (n * R1))
    efl_o, bfd_o = singlet().paraxial(lam)
    assert efl_o == pytest.approx(f, rel=1e-13)
    assert bfd_o == pytest.approx(bfd, rel=1e-13)


def test_image_plane_at_paraxial_focus():
    L = singlet()
    n = cauchy_n(LD)
    f = 1 / ((n - 1) * (2 / 50.0 - (n - 1) * 5.0 / (n * 2500.0)))
    bfd = f * (1 - (n - 1) * 5.0 / (n * 50.0))
    assert L.z_image() == pytest.approx(5.0 + bfd, rel=1e-13)


@pytest.mark.parametrize("lam", [400.0, LD, 700.0])
def test_exact_trace_reduces_to_paraxial_singlet(lam):
    """A ray at height h -> 0 parallel to the axis leaves with slope -h/EFL and
    crosses the axis at the back focal distance (aberrations are O(h^2))."""
    L = singlet()
    efl, bfd = L.paraxial(lam)
    h = 1e-4
    v, out, st = L.trace_states(h, 0.0, 0.0, 0.0, 1.0, lam)
    assert v == 1
    last = st[-2]                       # state right after surface 2
    slope = last[3] / last[5]
    assert slope == pytest.approx(-h / efl, rel=1e-6)
    z_cross = last[2] - last[0] / slope  # where the exit ray meets the axis
    assert z_cross - 5.0 == pytest.approx(bfd, rel=1e-6)


def paraxial_ynu(presc, lam, path=(0, 0), y0=1.0, u0=0.0):
    """Independent paraxial (y, n*u) raytrace of a path with the unfolded-mirror
    convention: a reflection turns the index to -n.  Returns (y, u) just after
    the last surface and the vertex z of that surface."""
    L = oracle.Lens(presc)
    S = presc.n_surfaces
    seq = oracle.path_sequence(S, *path)
    zv = presc.vertex_z()
    nm = [L.index(m, lam) for m in range(S + 1)]
    y, nu = y0, u0          # n*u with n = 1 in front
    n_cur = 1.0
    z_cur = zv[0] - presc.entrance_gap
    # start on the entrance plane: transfer to surface 1
    y = y + (zv[0] - z_cur) * u0
    z_cur = zv[0]
    first = True
    for s, typ, d in zip(*seq):
        if not first:
            dz = zv[s - 1] - z_cur           # signed axial travel
            y = y + dz * nu / n_cur          # n_cur is negative when travelling backward
        first = False
        z_cur = zv[s - 1]
        c = presc.surfaces[s - 1].curvature
        if typ == 0:
            n1 = nm[s - 1] if d > 0 else nm[s]
            n2 = nm[s] if d > 0 else nm[s - 1]
            n1s = n1 * d
            n2s = n2 * d
            nu = nu - y * (n2s - n1s) * c
            n_cur = n2s
        else:
            n1 = nm[s - 1] if d > 0 else nm[s]
            n1s = n1 * d
            n2s = -n1s
            nu = nu - y * (n2s - n1s) * c
            n_cur = n2s
    return y, nu / n_cur, z_cur


@pytest.mark.parametrize("path", [(0, 0), (1, 2)])
def test_exact_trace_reduces_to_paraxial_singlet_paths(path):
    L = singlet()
    p = w.singlet_lens()
    h = 1e-4
    y, u, z = paraxial_ynu(p, LD, path, y0=h)
    v, out, st = L.trace_states(h, 0.0, 0.0, 0.0, 1.0, LD, path=path)
    assert v == 1
    last = st[-2]
    assert last[0] == pytest.approx(y, rel=2e-6)
    assert last[3] / last[5] == pytest.approx(u, rel=2e-6)


def test_exact_trace_reduces_to_paraxial_eleven_main_and_ghosts(eleven):
    L = oracle.Lens(eleven)
    S = eleven.n_surfaces
    h = 1e-4
    for pid in [0, 1, 5, 17, 30, 54, 55]:
        path = oracle.path_ij(S, pid)
        y, u, z = paraxial_ynu(eleven, 550.0, path, y0=h)
        v, out, st = L.trace_states(h, 0.0, 0.0, 0.0, 1.0, 550.0, path=path)
        if v != 1:
            continue    # a ghost may leave the system backwards even paraxially
        last = st[-2]
        assert last[0] == pytest.approx(y, rel=1e-5, abs=1e-12), pid
        assert last[3] / last[5] == pytest.approx(u, rel=1e-5, abs=1e-12), pid


# ---------------------------------------------------------------- Fresnel

@pytest.mark.parametrize("n1,n2", [(1.0, 1.5167), (1.5167, 1.0), (1.62, 1.51), (1.0, 1.75)])
def test_fresnel_R_plus_T_from_amplitude_coefficients(n1, n2):
    """T computed from the transmission amplitudes (Hecht, Optics, Sec. 4.6)
    equals 1 - R at every angle below the critical angle."""
    for th in np.linspace(0.0, 1.5, 61):
        ci = math.cos(th)
        si = math.sin(th)
        if n1 * si / n2 >= 1.0:
            continue
        tir, Rs, Rp, ct = oracle.fresnel(n1, n2, ci)
        assert not tir
        ts = 2 * n1 * ci / (n1 * ci + n2 * ct)
        tp = 2 * n1 * ci / (n2 * ci + n1 * ct)
        f = (n2 * ct) / (n1 * ci)
        T = 0.5 * (f * ts * ts + f * tp * tp)
        assert 1.0 - 0.5 * (Rs + Rp) == pytest.approx(T, abs=1e-14)


def test_fresnel_normal_incidence():
    n = cauchy_n(LD)
    tir, Rs, Rp, ct = oracle.fresnel(1.0, n, 1.0)
    R0 = ((1 - n) / (1 + n)) ** 2
    assert Rs == pytest.approx(R0, rel=1e-14) and Rp == pytest.approx(R0, rel=1e-14)
    assert R0 == pytest.approx(0.0421599, abs=1e-7)


@pytest.mark.parametrize("n1,n2", [(1.0, 1.5167), (1.5167, 1.0)])
def test_fresnel_brewster(n1, n2):
    th = math.atan(n2 / n1)
    tir, Rs, Rp, ct = oracle.fresnel(n1, n2, math.cos(th))
    assert Rp < 1e-28
    assert Rs > 1e-3


def test_fresnel_critical_angle():
    n = 1.5167
    th_c = math.asin(1 / n)
    tir, Rs, Rp, ct = oracle.fresnel(n, 1.0, math.cos(th_c * (1 - 1e-7)))
    assert not tir and 0.5 * (Rs + Rp) > 0.99
    tir, Rs, Rp, ct = oracle.fresnel(n, 1.0, math.cos(th_c * (1 + 1e-7)))
    assert tir and Rs == 1.0 and Rp == 1.0


def test_snell_invariant_scalar():
    for n1, n2 in [(1.0, 1.6), (1.6, 1.0), (1.52, 1.71)]:
        for th in np.linspace(0.01, 1.4, 40):
            if n1 * math.sin(th) / n2 >= 1:
                continue
            tir, Rs, Rp, ct = oracle.fresnel(n1, n2, math.cos(th))
            assert n1 * math.sin(th) == pytest.approx(n2 * math.sqrt(1 - ct * ct), abs=1e-14)


# ---------------------------------------------------------------- on-axis closed forms

def test_on_axis_main_path_throughput():
    L = singlet()
    n = cauchy_n(LD)
    R0 = ((1 - n) / (1 + n)) ** 2
    v, out, e, k = L.trace_one(0.0, 0.0, 0.0, 0.0, 1.0, LD)
    assert v == 1
    assert out[5] == pytest.approx((1 - R0) ** 2, abs=1e-15)
    assert out[5] == pytest.approx(0.917458, abs=1e-6)
    assert out[0] == 0.0 and out[1] == 0.0 and out[4] == 1.0


def test_on_axis_ghost_throughput():
    L = singlet()
    n = cauchy_n(LD)
    R0 = ((1 - n) / (1 + n)) ** 2
    v, out, e, k = L.trace_one(0.0, 0.0, 0.0, 0.0, 1.0, LD, path=(1, 2))
    assert v == 1
    assert out[5] == pytest.approx((1 - R0) ** 2 * R0 ** 2, rel=1e-13)
    assert out[5] == pytest.approx(0.00163074, abs=1e-8)


# ---------------------------------------------------------------- plane-parallel plate

def plate(d=7.0, n=1.6, ap=30.0, zimg=40.0):
    g = w.Glass(kind=w.GLASS_CAUCHY, A=n, B=0.0)
    surfs = [w.Surface(0.0, d, ap, 0), w.Surface(0.0, 0.0, ap, -1)]
    return w.Prescription(surfaces=surfs, glasses=[g], entrance_gap=3.0, stop_after=0,
                          stop_offset=0.0, stop_r=0.0, image_mode=w.IMAGE_ABS, image_z=zimg)


@pytest.mark.parametrize("theta_deg", [0.0, 5.0, 20.0, 45.0])
def test_plate_closed_form(theta_deg):
    d, n, zimg = 7.0, 1.6, 40.0
    L = oracle.Lens(plate(d, n, zimg=zimg))
    th = math.radians(theta_deg)
    dx, dz = math.sin(th), math.cos(th)
    v, out, e, k = L.trace_one(0.5, 0.0, dx, 0.0, dz, 550.0)
    assert v == 1
    assert out[2] == pytest.approx(dx, abs=1e-15) and out[4] == pytest.approx(dz, abs=1e-15)
    shift = d * math.sin(th) * (1 - math.cos(th) / math.sqrt(n * n - math.sin(th) ** 2))
    x_expect = 0.5 + zimg * math.tan(th) - shift / math.cos(th)
    assert out[0] == pytest.approx(x_expect, abs=1e-12)
    tir, Rs, Rp, ct = oracle.fresnel(1.0, n, math.cos(th))
    R = 0.5 * (Rs + Rp)
    assert out[5] == pytest.approx((1 - R) ** 2, abs=1e-15)
    v, out, e, k = L.trace_one(0.5, 0.0, dx, 0.0, dz, 550.0, path=(1, 2))
    assert v == 1
    assert out[5] == pytest.approx((1 - R) ** 2 * R ** 2, rel=1e-12)
    assert out[2] == pytest.approx(dx, abs=1e-15)
    # the ghost crosses the plate three times; each leg inside advances x by
    # d * tan(theta_t), tan(theta_t) = sin(theta) / sqrt(n^2 - sin^2(theta))
    tan_t = math.sin(th) / math.sqrt(n * n - math.sin(th) ** 2)
    x_ghost = x_expect + 2 * d * tan_t
    assert out[0] == pytest.approx(x_ghost, abs=1e-12)


# ---------------------------------------------------------------- vector Snell on real surfaces

def test_hits_on_spheres_and_vector_snell(eleven):
    """Every recorded hit lies on its sphere; tangential n*d is conserved at a
    transmission and the normal component flips at a reflection (normals from
    the sphere centre, not from the oracle)."""
    L = oracle.Lens(eleven)
    S = eleven.n_surfaces
    zv = eleven.vertex_z()
    rays = w.eleven_rays(eleven, 300)
    checked = 0
    for pid in [0, 3, 20, 41]:
        path = oracle.path_ij(S, pid)
        surf, typ, dirs = oracle.path_sequence(S, *path)
        for r in range(len(rays)):
            ray = [a[r] for a in rays.arrays()]
            v, out, st = L.trace_states(*ray, path=path)
            nrec = len(st)
            lam = float(ray[5])
            nmed = [L.index(m, lam) for m in range(S + 1)]
            d_prev = np.array(ray[2:5], np.float64)
            d_prev /= np.linalg.norm(d_prev)
            for m in range(min(nrec, len(surf))):
                s, t, dr = surf[m], typ[m], dirs[m]
                p = st[m, 0:3]
                dn = st[m, 3:6]
                c = eleven.surfaces[s - 1].curvature
                R = 1.0 / c
                centre = np.array([0.0, 0.0, zv[s - 1] + R])
                assert abs(np.linalg.norm(p - centre) - abs(R)) < 1e-9 * abs(R)
                nv = (p - centre) / R      # unit normal (sign irrelevant below)
                n1 = nmed[s - 1] if dr > 0 else nmed[s]
                n2 = nmed[s] if dr > 0 else nmed[s - 1]
                tan_in = n1 * (d_prev - np.dot(d_prev, nv) * nv)
                if t == 0:
                    tan_out = n2 * (dn - np.dot(dn, nv) * nv)
                    assert np.allclose(tan_in, tan_out, atol=1e-12)
                    assert np.sign(np.dot(dn, nv)) == np.sign(np.dot(d_prev, nv))
                else:
                    tan_out = n1 * (dn - np.dot(dn, nv) * nv)
                    assert np.allclose(tan_in, tan_out, atol=1e-12)
                    assert np.dot(dn, nv) == pytest.approx(-np.dot(d_prev, nv), abs=1e-12)
                d_prev = dn
                checked += 1
    assert checked > 1000


# ---------------------------------------------------------------- reversibility

def reversed_prescription(p, z_image):
    """The mirror image z' = z_image - z of a prescription: surfaces in reverse
    order, curvatures negated, media reversed, stop gap g -> S - g."""
    S = p.n_surfaces
    zv = p.vertex_z()                                    # zv[k-1]: vertex of surface k
    media = [-1] + [s.glass_after for s in p.surfaces]   # medium m = 0..S
    media[S] = -1
    surfs = []
    zr = []
    for kp in range(1, S + 1):
        k = S + 1 - kp
        s = p.surfaces[k - 1]
        thick = zv[k - 1] - zv[k - 2] if k > 1 else 0.0
        surfs.append(w.Surface(-s.curvature, thick, s.aperture_r, media[k - 1]))
        zr.append(z_image - zv[k - 1])
    gp = S - p.stop_after
    zs = z_image - p.stop_z()
    off = zs - (0.0 if gp == 0 else zr[gp - 1])
    return w.Prescription(surfaces=surfs, glasses=copy.deepcopy(p.glasses),
                          entrance_gap=zr[0], stop_after=gp, stop_offset=off, stop_r=p.stop_r,
                          image_mode=w.IMAGE_ABS, image_z=z_image)


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_reversibility(which, eleven):
    p = w.singlet_lens() if which == "singlet" else eleven
    L = oracle.Lens(p)
    zi = L.z_image()
    Lr = oracle.Lens(reversed_prescription(p, zi))
    assert Lr.z_stop() == pytest.approx(zi - L.z_stop(), abs=1e-12)
    rays = w.singlet_rays(400) if which == "singlet" else w.eleven_rays(p, 400)
    n_ok = 0
    for r in range(len(rays)):
        ray = [float(a[r]) for a in rays.arrays()]
        v, out, e, k = L.trace_one(*ray)
        if v != 1 or e < 1e-6:
            continue
        v2, back, e2, k2 = Lr.trace_one(out[0], out[1], -out[2], -out[3], out[4], ray[5])
        assert v2 == 1
        d0 = np.array(ray[2:5]) / np.linalg.norm(ray[2:5])
        assert back[0] == pytest.approx(ray[0], abs=1e-9)
        assert back[1] == pytest.approx(ray[1], abs=1e-9)
        assert back[2] == pytest.approx(-d0[0], abs=1e-11)
        assert back[3] == pytest.approx(-d0[1], abs=1e-11)
        assert back[5] == pytest.approx(out[5], rel=1e-11)
        n_ok += 1
    assert n_ok > 50


# ---------------------------------------------------------------- symmetry (paper Sec. 4.1, Eq. 10)

@pytest.mark.parametrize("pid", [0, 7, 33])
def test_rotation_and_mirror_equivariance(eleven, pid):
    L = oracle.Lens(eleven)
    path = oracle.path_ij(eleven.n_surfaces, pid)
    rays = w.eleven_rays(eleven, 400)
    rng = np.random.default_rng(3)
    for r in range(len(rays)):
        x, y, dx, dy, dz, lam = [float(a[r]) for a in rays.arrays()]
        v, out, e, k = L.trace_one(x, y, dx, dy, dz, lam, path=path)
        if e < 1e-6:
            continue
        phi = rng.uniform(0, 2 * math.pi)
        c, s = math.cos(phi), math.sin(phi)
        v2, out2, e2, k2 = L.trace_one(c * x - s * y, s * x + c * y, c * dx - s * dy,
                                       s * dx + c * dy, dz, lam, path=path)
        assert v2 == v
        if v == 1:
            assert out2[0] == pytest.approx(c * out[0] - s * out[1], abs=1e-10)
            assert out2[1] == pytest.approx(s * out[0] + c * out[1], abs=1e-10)
            assert out2[2] == pytest.approx(c * out[2] - s * out[3], abs=1e-12)
            assert out2[5] == pytest.approx(out[5], rel=1e-12)
        v3, out3, e3, k3 = L.trace_one(x, -y, dx, -dy, dz, lam, path=path)
        assert v3 == v
        if v == 1:
            assert out3[1] == pytest.approx(-out[1], abs=1e-12)
            assert out3[0] == pytest.approx(out[0], abs=1e-12)
            assert out3[5] == pytest.approx(out[5], rel=1e-13)


# ---------------------------------------------------------------- tiny brute-force cases

def test_aperture_is_a_closed_disc():
    p = plate(ap=4.0)
    p.surfaces[0].aperture_r = 4.0
    L = oracle.Lens(p)
    v, out, e, k = L.trace_one(4.0, 0.0, 0.0, 0.0, 1.0, 550.0)
    assert v == 1 and e == 0.0
    v, out, e, k = L.trace_one(math.nextafter(4.0, 5.0), 0.0, 0.0, 0.0, 1.0, 550.0)
    assert v == 0


def test_stop_blocks_and_passes_singlet():
    L = singlet()
    # inside the 10 mm stop, parallel: passes
    assert L.trace_one(9.9, 0.0, 0.0, 0.0, 1.0, 550.0)[0] == 1
    # outside the stop at the entrance plane: blocked by the stop alone
    v, out, e, k = L.trace_one(10.05, 0.0, -0.1, 0.0, math.sqrt(1 - 0.01), 550.0)
    assert v == 0 and e == pytest.approx(0.05, abs=1e-12)
    # inside the stop but leaving the clear aperture of surface 2
    v, out, e, k = L.trace_one(9.5, 0.0, 0.3, 0.0, math.sqrt(1 - 0.09), 550.0)
    assert v == 0


def test_ray_missing_the_sphere_is_invalid():
    # a steep ray that never meets a strongly curved surface
    g = w.Glass(kind=w.GLASS_CAUCHY, A=1.5, B=0.0)
    p = w.Prescription(surfaces=[w.Surface(1 / 5.0, 2.0, 4.9, 0), w.Surface(0.0, 0.0, 20.0, -1)],
                       glasses=[g], entrance_gap=1.0, image_mode=w.IMAGE_ABS, image_z=30.0)
    L = oracle.Lens(p)
    v, out, e, k = L.trace_one(0.0, 8.0, 0.0, 0.0, 1.0, 550.0)
    assert v == 0


def test_bad_inputs_flagged():
    L = singlet()
    assert L.trace_one(float("nan"), 0, 0, 0, 1, 550.0)[0] == -1
    assert L.trace_one(0, 0, 0, 0, -1, 550.0)[0] == -1
    assert L.trace_one(0, 0, 0, 0, 1, 0.0)[0] == -1


def test_ghost_leaving_backwards_is_invalid():
    L = singlet()
    # strong ghost geometry: a ray that reflects back out of the entrance is not valid
    v, out, e, k = L.trace_one(0.0, 0.0, 0.0, 0.0, 1.0, LD, path=(1, 2))
    assert v == 1
    assert L.trace_one(0, 0, 0, 0, 1, LD, path=(2, 1))[0] == -1


# ---------------------------------------------------------------- dispersion

def test_sellmeier_matches_catalogue_bk7():
    """N-BK7 Sellmeier coefficients (Schott catalogue) give the catalogue
    n_d = 1.51680 and n_F, n_C to 1e-5."""
    g = w.Glass(kind=w.GLASS_SELLMEIER, A=0, B=0, B3=(1.03961212, 0.231792344, 1.01046945),
                C3=(0.00600069867, 0.0200179144, 103.560653))
    p = w.Prescription(surfaces=[w.Surface(0.0, 5.0, 10.0, 0), w.Surface(0.0, 0.0, 10.0, -1)],
                       glasses=[g], image_mode=w.IMAGE_ABS, image_z=20.0)
    L = oracle.Lens(p)
    assert L.index(1, 587.5618) == pytest.approx(1.51680, abs=1e-5)
    assert L.index(1, 486.1327) == pytest.approx(1.52238, abs=1e-5)
    assert L.index(1, 656.2725) == pytest.approx(1.51432, abs=1e-5)
    assert L.index(0, 500.0) == 1.0


# ---------------------------------------------------------------- path codes (paper Fig. 7)

def test_path_codes_from_paper_figure():
    """The flare paths the paper names (Fig. 7 caption): 131092 and 65616.
    Reading: LSB = first interaction, leading sentinel 1; the 59 mm lens path
    is ghost (1, 3) of 13 interfaces and the 22 mm lens path ghost (3, 5) of 12."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "path_codes.json")))
    for case in gold["cases"]:
        assert oracle.path_code(case["S"], case["i"], case["j"]) == case["code"]


def test_path_sequence_counts():
    for S in [2, 5, 11]:
        assert len(oracle.path_sequence(S, 0, 0)[0]) == S
        for i in range(1, S + 1):
            for j in range(i + 1, S + 1):
                surf, typ, d = oracle.path_sequence(S, i, j)
                assert len(surf) == S + 2 * (j - i)
                assert sum(typ) == 2
                assert surf[j - 1] == j and typ[j - 1] == 1
                assert surf[2 * j - i - 1] == i and typ[2 * j - i - 1] == 1
        ids = [oracle.path_ij(S, k) for k in range(1, S * (S - 1) // 2 + 1)]
        assert len(set(ids)) == S * (S - 1) // 2


def test_throughput_is_the_amplitude_fresnel_product_along_paths(eleven):
    """At every interface a traced ray meets, the oracle's throughput changes
    by the transmittance (n2 cos t)/(n1 cos i) (t_s^2 + t_p^2)/2 or by the
    reflectance (r_s^2 + r_p^2)/2 of the textbook amplitude coefficients
    (Hecht, Optics, Sec. 4.6), recomputed here from the recorded hit, the
    sphere's centre and Snell's law; the two add to 1 at each interface."""
    L = oracle.Lens(eleven)
    S = eleven.n_surfaces
    zv = eleven.vertex_z()
    rays = w.eleven_rays(eleven, 200)
    checked = reflections = 0
    for pid in [0, 5, 30, 54]:
        path = oracle.path_ij(S, pid)
        surf, typ, dirs = oracle.path_sequence(S, *path)
        for r in range(len(rays)):
            ray = [float(a[r]) for a in rays.arrays()]
            v, out, st = L.trace_states(*ray, path=path)
            lam = ray[5]
            nmed = [L.index(m, lam) for m in range(S + 1)]
            d_prev = np.array(ray[2:5], np.float64)
            d_prev /= np.linalg.norm(d_prev)
            I_prev = 1.0
            for m in range(min(len(st), len(surf))):
                s, t, dr = surf[m], typ[m], dirs[m]
                p, dn, I = st[m, 0:3], st[m, 3:6], st[m, 6]
                R = 1.0 / eleven.surfaces[s - 1].curvature
                nv = (p - np.array([0.0, 0.0, zv[s - 1] + R])) / R
                n1 = nmed[s - 1] if dr > 0 else nmed[s]
                n2 = nmed[s] if dr > 0 else nmed[s - 1]
                ci = abs(float(np.dot(d_prev, nv)))
                sin_t = n1 / n2 * math.sqrt(max(0.0, 1.0 - ci * ci))
                if sin_t >= 1.0:
                    assert t == 1 and I == pytest.approx(I_prev, rel=1e-12)   # total reflection
                else:
                    ct = math.sqrt(1.0 - sin_t * sin_t)
                    if t == 0:
                        assert abs(float(np.dot(dn, nv))) == pytest.approx(ct, abs=1e-12)
                    ts = 2 * n1 * ci / (n1 * ci + n2 * ct)
                    tp = 2 * n1 * ci / (n2 * ci + n1 * ct)
                    rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct)
                    rp = (n2 * ci - n1 * ct) / (n2 * ci + n1 * ct)
                    Tamp = n2 * ct / (n1 * ci) * 0.5 * (ts * ts + tp * tp)
                    Ramp = 0.5 * (rs * rs + rp * rp)
                    assert Tamp + Ramp == pytest.approx(1.0, abs=1e-12)
                    assert I == pytest.approx(I_prev * (Tamp if t == 0 else Ramp), rel=1e-11)
                reflections += t == 1
                I_prev, d_prev = I, dn
                checked += 1
            if v == 1:
                assert out[5] == pytest.approx(I_prev, rel=1e-12)
    assert checked > 1000 and reflections > 50
