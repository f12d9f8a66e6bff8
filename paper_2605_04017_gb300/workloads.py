"""Seeded synthetic workloads: lens prescriptions, entrance rays, wavelengths.

This module is shared by the CUDA path's tests and benchmark and by the
CPU oracle's tests.  It holds no arithmetic of the method itself (no
intersection, refraction, Fresnel, paraxial or map code): it only draws
random numbers and lays out inputs.  Where a generated lens must pass a
check that needs optics (a positive focal length), the caller supplies
that check as ``accept``.

Frame (paper Sec. 3): the optical axis is +z, light enters travelling +z,
the entrance plane is z = 0, surface 1's vertex is at ``entrance_gap``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

GLASS_AIR = 0
GLASS_CAUCHY = 1
GLASS_SELLMEIER = 2

IMAGE_PARAXIAL = 0
IMAGE_ABS = 1

LAMBDA_D_NM = 587.6          # helium d line, the reference wavelength
LAMBDA_LO_NM = 380.0
LAMBDA_HI_NM = 780.0
SEED_BASE = 20260504         # config k draws from SEED_BASE + k


@dataclasses.dataclass
class Glass:
    """One glass.  Cauchy: n = A + B / lam^2; Sellmeier: n^2 = 1 + sum B_i lam^2/(lam^2 - C_i).

    Wavelengths in micrometres.
    """
    kind: int = GLASS_CAUCHY
    A: float = 1.5
    B: float = 0.0
    B3: Sequence[float] = (0.0, 0.0, 0.0)
    C3: Sequence[float] = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class Surface:
    curvature: float      # 1/R in 1/mm, 0 = plane; R > 0 means centre of curvature at +z
    thickness: float      # vertex-to-next-vertex distance in mm
    aperture_r: float     # clear aperture radius in mm
    glass_after: int      # index into Prescription.glasses of the medium after this surface, -1 = air
    conic: float = 0.0    # even asphere: conic constant kappa (0 with zero asph: a sphere)
    asph: tuple = (0.0, 0.0, 0.0, 0.0)   # even asphere: A4, A6, A8, A10 (mm^-3, mm^-5, ...)


@dataclasses.dataclass
class Prescription:
    surfaces: List[Surface]
    glasses: List[Glass]
    entrance_gap: float = 0.0     # entrance plane (z=0) to surface-1 vertex, mm
    stop_after: int = 0           # stop lies in the gap after this surface (0: before surface 1)
    stop_offset: float = 0.0      # stop plane z relative to that gap's start plane (z=0 or vertex k)
    stop_r: float = 0.0           # stop radius; <= 0 means no stop
    image_mode: int = IMAGE_PARAXIAL
    image_z: float = 0.0          # absolute image-plane z when image_mode == IMAGE_ABS
    lambda_ref_nm: float = LAMBDA_D_NM

    @property
    def n_surfaces(self) -> int:
        return len(self.surfaces)

    def vertex_z(self) -> np.ndarray:
        z = [self.entrance_gap]
        for s in self.surfaces[:-1]:
            z.append(z[-1] + s.thickness)
        return np.asarray(z, dtype=np.float64)

    def stop_z(self) -> float:
        base = 0.0 if self.stop_after == 0 else float(self.vertex_z()[self.stop_after - 1])
        return base + self.stop_offset


# --------------------------------------------------------------------------------------
# Lenses
# --------------------------------------------------------------------------------------

def singlet_lens() -> Prescription:
    """The 2-surface singlet: R1 = +50 mm, R2 = -50 mm, 5 mm thick, clear radius 10 mm,
    stop (radius 10 mm) at the front vertex, Cauchy glass n = 1.5046 + 0.00420/lam^2,
    image plane at the paraxial focus for the d line."""
    g = Glass(kind=GLASS_CAUCHY, A=1.5046, B=0.00420)
    surfs = [Surface(1.0 / 50.0, 5.0, 10.0, 0), Surface(-1.0 / 50.0, 0.0, 10.0, -1)]
    return Prescription(surfaces=surfs, glasses=[g], entrance_gap=0.0, stop_after=0,
                        stop_offset=0.0, stop_r=10.0, image_mode=IMAGE_PARAXIAL)


def _sag(c: float, r: np.ndarray) -> np.ndarray:
    # Input geometry only (shape of a generated surface), used to reject
    # overlapping draws; the method's intersection code lives elsewhere.
    return c * r * r / (1.0 + np.sqrt(np.maximum(0.0, 1.0 - c * c * r * r)))


def glass_pattern(S: int) -> List[bool]:
    """Which media after surfaces 1..S are glass (True) or air (False).

    Alternating singlets; an odd surface count gets one cemented doublet,
    placed right after the stop gap (for S = 11: G A G A G A | G G A G A).
    The medium after surface S is always air.
    """
    if S < 2:
        raise ValueError("need at least 2 surfaces")
    n_single = S // 2 if S % 2 == 0 else (S - 3) // 2
    # media list built element by element
    elems: List[int] = [2] * n_single           # 2 surfaces per singlet
    if S % 2 == 1:
        front = n_single // 2 + 1                 # singlets in front of the stop
        elems = [2] * front + [3] + [2] * (n_single - front)
    pat: List[bool] = []
    for e in elems:
        pat += [True] * (e - 1) + [False]
    assert len(pat) == S and not pat[-1]
    return pat


def stop_gap_index(pattern: List[bool]) -> int:
    """The middle air gap between elements: returns k such that the stop lies after surface k."""
    gaps = [k + 1 for k in range(len(pattern) - 1) if not pattern[k]]
    if not gaps:
        return 0
    if len(pattern) % 2 == 1:
        # the cemented doublet follows the stop: the gap in front of it
        n_single = (len(pattern) - 3) // 2
        front = n_single // 2 + 1
        return 2 * front
    return gaps[(len(gaps) - 1) // 2]


def generate_lens(seed: int, S: int, accept: Callable[[Prescription], bool],
                  r_range=(20.0, 200.0), t_range=(1.0, 8.0), a_range=(8.0, 15.0),
                  A_range=(1.48, 1.75), B_range=(0.003, 0.012), clearance=0.5,
                  max_tries=10000) -> Prescription:
    """Seeded random rotationally symmetric lens of S spherical surfaces.

    |R| ~ U[r_range] with a random sign, thickness ~ U[t_range], aperture
    ~ U[a_range], one Cauchy (A, B) per glass element, stop radius = the
    smaller neighbouring aperture, stop centred in the middle air gap.  A gap is
    redrawn until the two surfaces stay ``clearance`` mm apart over the
    smaller aperture and the stop plane clears both sags; a whole lens is
    redrawn until ``accept(lens)`` is true (the caller's focal-length check).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pat = glass_pattern(S)
    kstop = stop_gap_index(pat)
    for _ in range(max_tries):
        curv = []
        for _k in range(S):
            R = rng.uniform(*r_range) * (1.0 if rng.uniform() < 0.5 else -1.0)
            curv.append(1.0 / R)
        ap = [float(rng.uniform(*a_range)) for _ in range(S)]
        # one glass per glass medium (the two halves of a cemented pair differ)
        glasses: List[Glass] = []
        gidx: List[int] = []
        for k in range(S):
            if pat[k]:
                glasses.append(Glass(GLASS_CAUCHY, float(rng.uniform(*A_range)),
                                     float(rng.uniform(*B_range))))
                gidx.append(len(glasses) - 1)
            else:
                gidx.append(-1)
        thick = []
        ok = True
        for k in range(S - 1):
            amin = min(ap[k], ap[k + 1])
            rr = np.linspace(0.0, amin, 33)
            for _t in range(1000):
                t = float(rng.uniform(*t_range))
                gap = t + _sag(curv[k + 1], rr) - _sag(curv[k], rr)
                good = bool(np.all(gap >= clearance))
                if good and k + 1 == kstop:
                    a_s = amin
                    zs = 0.5 * t
                    lo = float(np.max(_sag(curv[k], np.linspace(0, a_s, 33))))
                    hi = t + float(np.min(_sag(curv[k + 1], np.linspace(0, a_s, 33))))
                    good = (lo + clearance <= zs <= hi - clearance)
                if good:
                    break
            else:
                ok = False
                break
            thick.append(t)
        if not ok:
            continue
        thick.append(0.0)
        surfs = [Surface(curv[k], thick[k], ap[k], gidx[k]) for k in range(S)]
        sag1 = float(_sag(curv[0], np.array([ap[0]]))[0])
        entrance_gap = 2.0 + max(0.0, -sag1)
        if kstop > 0:
            stop_r = min(ap[kstop - 1], ap[kstop])
            stop_off = 0.5 * thick[kstop - 1]
        else:
            stop_r = ap[0]
            stop_off = 0.5 * entrance_gap
        lens = Prescription(surfaces=surfs, glasses=glasses, entrance_gap=entrance_gap,
                            stop_after=kstop, stop_offset=stop_off, stop_r=stop_r,
                            image_mode=IMAGE_PARAXIAL)
        if accept(lens):
            return lens
    raise RuntimeError("generate_lens: no acceptable lens found")


# --------------------------------------------------------------------------------------
# Rays
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Rays:
    """SoA FP32 entrance rays on the plane z = 0 plus wavelengths in nm."""
    x: np.ndarray
    y: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    lam: np.ndarray

    def __len__(self) -> int:
        return int(self.x.shape[0])

    def arrays(self):
        return [self.x, self.y, self.dx, self.dy, self.dz, self.lam]

    def subset(self, idx) -> "Rays":
        return Rays(*[a[idx].copy() for a in self.arrays()])


def entrance_rays(n: int, seed: int, rho: float, half_angle_deg: float = 10.0,
                  lam_range=(LAMBDA_LO_NM, LAMBDA_HI_NM)) -> Rays:
    """Positions uniform on a disk of radius ``rho``; direction angles theta_x, theta_y
    independently uniform in +-half_angle; d = normalize(tan theta_x, tan theta_y, 1);
    wavelength uniform in lam_range.  Drawn in FP64, stored as FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rho * np.sqrt(rng.uniform(size=n))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    h = math.radians(half_angle_deg)
    tx = np.tan(rng.uniform(-h, h, size=n))
    ty = np.tan(rng.uniform(-h, h, size=n))
    lam = rng.uniform(lam_range[0], lam_range[1], size=n)
    inv = 1.0 / np.sqrt(tx * tx + ty * ty + 1.0)
    f = np.float32
    return Rays(x=(r * np.cos(phi)).astype(f), y=(r * np.sin(phi)).astype(f),
                dx=(tx * inv).astype(f), dy=(ty * inv).astype(f), dz=inv.astype(f),
                lam=lam.astype(f))


def redraw_wavelengths(n: int, seed: int, lam_range=(LAMBDA_LO_NM, LAMBDA_HI_NM)) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lam_range[0], lam_range[1], size=n).astype(np.float32)


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------

SINGLET_RHO = 12.0          # entrance disk radius for the singlet (radius, not diameter)
SINGLET_N = 65536
ELEVEN_N = 4194304
ELEVEN_FIT_N = 16777216
PRECISION_N = 16777216
FLARE_N_PER_PATH = 1048576


def eleven_surface_lens(accept: Callable[[Prescription], bool]) -> Prescription:
    """The seeded 11-surface double-Gauss-like lens."""
    return generate_lens(SEED_BASE + 2, 11, accept)


def eleven_rho(lens: Prescription) -> float:
    return 1.2 * lens.surfaces[0].aperture_r


def singlet_rays(n: int = SINGLET_N) -> Rays:
    return entrance_rays(n, SEED_BASE + 1, SINGLET_RHO)


def eleven_rays(lens: Prescription, n: int = ELEVEN_N) -> Rays:
    return entrance_rays(n, SEED_BASE + 2, eleven_rho(lens))


def eleven_fit_rays(lens: Prescription, n: int = ELEVEN_FIT_N) -> Rays:
    return entrance_rays(n, SEED_BASE + 2 + 1000, eleven_rho(lens))


def precision_rays(n: int = PRECISION_N) -> Rays:
    return entrance_rays(n, SEED_BASE + 3, SINGLET_RHO)


def flare_rays(lens: Prescription, n: int = FLARE_N_PER_PATH) -> Rays:
    return entrance_rays(n, SEED_BASE + 4, eleven_rho(lens))


def flare_wavelengths(path_id: int, n: int = FLARE_N_PER_PATH) -> np.ndarray:
    return redraw_wavelengths(n, SEED_BASE + 4 + path_id)


def serving_lenses(accept: Callable[[Prescription], bool], count: int = 8) -> List[Prescription]:
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 5))
    out = []
    for k in range(count):
        S = int(rng.integers(4, 23))
        out.append(generate_lens(SEED_BASE + 5 + 100 * (k + 1), S, accept))
    return out


def xavier_uniform(fan_in: int, fan_out: int, rng: np.random.Generator) -> np.ndarray:
    """Xavier-uniform draw of a fan_out x fan_in weight matrix (FP64)."""
    lim = math.sqrt(6.0 / (fan_in + fan_out))
    return rng.uniform(-lim, lim, size=(fan_out, fan_in))
