"""ORACLE -- test infrastructure only (see oracle/__init__.py).

The lens seen from its image side, for backward path tracing (Sec. 3,
Eq. 9: rays leave the sensor, cross the lens in reverse along the full
transmission path and continue into the scene).  Reading: the backward
transport of a lens is the forward transport of its mirror image about the
sensor plane.  With z' = sensor_z - z:
  - surface j of the reversed lens is forward surface k = S + 1 - j, at
    z'_j = sensor_z - z_k, with curvature -c_k and, for an even asphere,
    polynomial coefficients -A_k (mirroring flips the sag; the conic
    constant stays), and the same clear aperture;
  - the medium after reversed surface j is the forward medium in front of
    surface k (air for k = 1);
  - the reversed entrance plane (z' = 0) is the sensor, and its output
    plane is z' = sensor_z - out_z, a plane in front of forward surface 1;
  - the stop keeps its plane and radius.
A ray leaving the sensor at (x, y) towards the lens along the forward
direction (dx, dy, -dz), dz > 0, is the reversed-frame ray (x, y, dx, dy,
dz); an output (x', y', dx', dy', dz') is the forward-frame ray at z = out_z
travelling along (dx', dy', -dz').

Parity status: pinned by reversibility (a forward trace followed by the
backward trace of its reversed exit ray returns to the entrance ray, with
the same throughput), by the reversed lens's effective focal length (equal
to the forward one), and by double reversal.
"""
from __future__ import annotations

import dataclasses


def vertex_z(presc):
    """Forward vertex z of surfaces 1..S (entrance plane at z = 0)."""
    z = [presc.entrance_gap]
    for s in presc.surfaces[:-1]:
        z.append(z[-1] + s.thickness)
    return z


def stop_z(presc):
    zv = vertex_z(presc)
    base = 0.0 if presc.stop_after == 0 else zv[presc.stop_after - 1]
    return base + presc.stop_offset


def reverse_prescription(presc, sensor_z: float, out_z: float, image_abs_mode: int):
    """The reversed prescription (same types as `presc`); image_abs_mode is the
    prescription's code for an absolute image plane."""
    S = len(presc.surfaces)
    zv = vertex_z(presc)                 # zv[k - 1] = z of forward surface k
    surf_t = type(presc.surfaces[0])
    surfs = []
    for j in range(1, S + 1):
        k = S + 1 - j
        s = presc.surfaces[k - 1]
        thick = zv[k - 1] - zv[k - 2] if k >= 2 else 0.0
        glass = presc.surfaces[k - 2].glass_after if k >= 2 else -1
        # mirroring negates the sag: the curvature and the polynomial terms change
        # sign, the conic constant does not
        surfs.append(surf_t(curvature=-s.curvature, thickness=thick, aperture_r=s.aperture_r,
                            glass_after=glass, conic=getattr(s, "conic", 0.0),
                            asph=tuple(-a for a in getattr(s, "asph", (0.0, 0.0, 0.0, 0.0)))))
    stop_after, stop_offset = 0, 0.0
    if presc.stop_r > 0.0:
        g = presc.stop_after               # forward gap between vertex g and g + 1 (vertex 0: z = 0)
        zs = stop_z(presc)
        stop_after = S - g
        if stop_after == 0:                # forward stop behind the last surface
            stop_offset = sensor_z - zs
        else:                              # relative to reversed surface S - g = forward surface g + 1
            stop_offset = zv[g] - zs
    return dataclasses.replace(presc, surfaces=surfs, entrance_gap=sensor_z - zv[S - 1],
                               stop_after=stop_after, stop_offset=stop_offset,
                               image_mode=image_abs_mode, image_z=sensor_z - out_z)
