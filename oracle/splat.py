"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Forward light tracing onto the sensor, Sec. 3, Eq. 8: the image a set of
entrance rays produces is the sum, over every path P and every ray whose
path is valid, of the path's output throughput I_out times the projected
geometric factor G times the pixel filter h evaluated at the ray's sensor
hit x_out.  Readings (the paper names neither h nor G's form):
  - G is the cosine between the exit direction and the sensor normal (+z),
    i.e. d_z of the exit direction -- the paper's pipeline listing weights
    each deposit by the dot product of the exit direction with the sensor
    normal;
  - h is the tent (bilinear) filter of one pixel radius,
    h(p - c) = max(0, 1 - |p_x - c_x| / s) * max(0, 1 - |p_y - c_y| / s),
    s the pixel side, c a pixel centre;
  - the sensor is a W x H grid of square pixels centred on the axis:
    pixel (i, j) has its centre at ((i + 0.5 - W / 2) s, (j + 0.5 - H / 2) s);
  - every deposit is scaled by a constant `weight` (1 / rays for the
    per-sample average of the pipeline listing).
FP64 throughout.  Two formulations are given: `splat`, which finds a
ray's (at most four) pixels from its continuous pixel coordinate, and
`splat_brute`, which evaluates h at every pixel centre; the tests pin one
against the other and against hand-computed cases.

Parity status: pinned (hand cases, brute force, weight conservation).
"""
from __future__ import annotations

import numpy as np


def pixel_coords(x, y, width: int, height: int, pixel_mm: float):
    """Continuous pixel coordinates (u, v): pixel (i, j)'s centre is at (i, j)."""
    u = np.asarray(x, np.float64) / pixel_mm + width / 2.0 - 0.5
    v = np.asarray(y, np.float64) / pixel_mm + height / 2.0 - 0.5
    return u, v


def splat(x, y, dz, I, valid, width: int, height: int, pixel_mm: float, weight: float = 1.0,
          image=None):
    """Accumulate Eq. 8's deposits of rays with valid != 0 into image[height, width]
    (FP64; created zero when None) and return it."""
    if image is None:
        image = np.zeros((height, width), np.float64)
    valid = np.asarray(valid) != 0
    u, v = pixel_coords(np.asarray(x)[valid], np.asarray(y)[valid], width, height, pixel_mm)
    w = np.asarray(I, np.float64)[valid] * np.asarray(dz, np.float64)[valid] * weight
    i0 = np.floor(u)
    j0 = np.floor(v)
    fx = u - i0
    fy = v - j0
    i0 = i0.astype(np.int64)
    j0 = j0.astype(np.int64)
    for di, wx in ((0, 1.0 - fx), (1, fx)):
        for dj, wy in ((0, 1.0 - fy), (1, fy)):
            ii = i0 + di
            jj = j0 + dj
            ok = (ii >= 0) & (ii < width) & (jj >= 0) & (jj < height)
            np.add.at(image, (jj[ok], ii[ok]), (w * wx * wy)[ok])
    return image


def splat_brute(x, y, dz, I, valid, width: int, height: int, pixel_mm: float, weight: float = 1.0):
    """The same sum with h evaluated at every pixel centre of the sensor
    (slow; for small sensors and few rays)."""
    image = np.zeros((height, width), np.float64)
    ci = (np.arange(width) + 0.5 - width / 2.0) * pixel_mm
    cj = (np.arange(height) + 0.5 - height / 2.0) * pixel_mm
    for r in range(len(x)):
        if not valid[r]:
            continue
        hx = np.maximum(0.0, 1.0 - np.abs(float(x[r]) - ci) / pixel_mm)
        hy = np.maximum(0.0, 1.0 - np.abs(float(y[r]) - cj) / pixel_mm)
        image += float(I[r]) * float(dz[r]) * weight * np.outer(hy, hx)
    return image


def deposit_bound(x, y, dz, I, valid, width: int, height: int, pixel_mm: float, weight: float,
                  pos_tol: float, val_tol: float):
    """Per-pixel bound on how far a splat of the same rays can move when each
    ray's sensor hit is off by at most pos_tol (mm) per axis and each of I and
    d_z by at most val_tol: sum over the rays touching the pixel (with the
    footprint widened by pos_tol) of weight * (I dz (|du| + |dv|) + (I + dz) val_tol),
    du = dv = pos_tol / pixel_mm (the tent's slope is 1 / pixel per axis)."""
    image = np.zeros((height, width), np.float64)
    valid = np.asarray(valid) != 0
    xs, ys = np.asarray(x, np.float64)[valid], np.asarray(y, np.float64)[valid]
    d = pos_tol / pixel_mm
    w = (np.abs(np.asarray(I, np.float64)[valid] * np.asarray(dz, np.float64)[valid]) * 2.0 * d +
         (np.abs(np.asarray(I, np.float64)[valid]) + np.abs(np.asarray(dz, np.float64)[valid])) * val_tol) * weight
    u, v = pixel_coords(xs, ys, width, height, pixel_mm)
    for du in (-d, d):
        for dv in (-d, d):
            i0 = np.floor(u + du).astype(np.int64)
            j0 = np.floor(v + dv).astype(np.int64)
            for di in (0, 1):
                for dj in (0, 1):
                    ii, jj = i0 + di, j0 + dj
                    ok = (ii >= 0) & (ii < width) & (jj >= 0) & (jj < height)
                    # max over the corners of the widened footprint: add, then the
                    # caller's comparison is conservative (a pixel counted up to 4x)
                    np.add.at(image, (jj[ok], ii[ok]), w[ok])
    return image
