"""ORACLE -- test infrastructure only.

Plain, slow, obviously-correct CPU reference for the lens-transport hot
path (paper: Precomputed Lens Transport Maps, Sec. 3 Eq. 1-7, Sec. 4.2,
Sec. 5.1).  The tracer and the tabulated map are single-threaded FP64 C
(``trace.c``, ``map.c``); the learned networks (``mlp.py``) and the
polynomial-patch map (``poly.py``) are FP64 numpy.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline (its ``cpu_baseline`` object and its ``--impl reference`` arm) may
import this package.  It shares no code with the CUDA library and never
imports it.

Parity status per function (what pins it; see tests/test_oracle_*.py):
  or_trace       paraxial ABCD/lensmaker focal lengths, Fresnel closed forms,
                 plate closed form, Snell invariant, reversibility, symmetry,
                 hand-enumerated tiny cases, the paper's path codes; even
                 aspheres: the zero-asphere sphere, a Cartesian oval's
                 perfect focus, a polynomial surface's hit and normal
  or_map_*       affine-field exactness, node reproduction, brute-force class
  quantize16     exact round trip of representable values, the half-step
                 error bound, the exponent's bracket, zeros for invalid
                 nodes, the quantised query within half a step of the FP64 one
  poly           polynomial-patch map: exact reproduction of degree-<=D fields
                 (and not of degree D + 1), the symmetry reduction's rotation
                 invariance and round trip, unclipped = real lens on valid
                 rays, brute-force classes, the exact trace within the
                 certified residual
  mlp            finite differences, closed-form tiny networks, Adam step
  splat          pixel-centre, pixel-corner and quarter-offset deposits,
                 brute-force tent filter, conservation of weight, symmetry
  mcmc           SplitMix64 reference outputs, the uniform stationary law
                 over the valid region, chain invariants
  reverse        a backward trace returns to the entrance ray, equal focal
                 lengths from both sides, the stop keeps its plane
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["trace.c", "map.c"]
_LIB: Optional[ctypes.CDLL] = None
_LOCK = threading.Lock()


def _so_path() -> str:
    return os.path.join(_HERE, "_build", "liblt_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no FMA contraction, no fast-math)."""
    out = _so_path()
    srcs = [os.path.join(_HERE, s) for s in _SRCS] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SRCS] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib() -> ctypes.CDLL:
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = ctypes.CDLL(build())
            _declare(_LIB)
    return _LIB


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)
_bp = ctypes.POINTER(ctypes.c_ubyte)


def _declare(L: ctypes.CDLL) -> None:
    L.or_lens_sizeof.restype = ctypes.c_int
    L.or_lens_init.restype = ctypes.c_int
    L.or_lens_init.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp, _ip, ctypes.c_int, _ip,
                               _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.or_lens_set_asphere.restype = ctypes.c_int
    L.or_lens_set_asphere.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
    L.or_lens_get.restype = ctypes.c_double
    L.or_lens_get.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.or_index.restype = ctypes.c_double
    L.or_index.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
    L.or_paraxial.restype = ctypes.c_int
    L.or_paraxial.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp]
    L.or_fresnel.restype = ctypes.c_int
    L.or_fresnel.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
    L.or_path_sequence.restype = ctypes.c_int
    L.or_path_sequence.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip, _ip]
    L.or_path_code.restype = ctypes.c_ulonglong
    L.or_path_code.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.or_path_ij.restype = ctypes.c_int
    L.or_path_ij.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip]
    L.or_trace_one.restype = ctypes.c_int
    L.or_trace_one.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int] + \
        [ctypes.c_double] * 6 + [_dp, _dp, _dp]
    L.or_trace_states.restype = ctypes.c_int
    L.or_trace_states.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int] + \
        [ctypes.c_double] * 6 + [_dp, _dp, _ip]
    L.or_trace.restype = ctypes.c_long
    L.or_trace.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_long] + \
        [_fp] * 6 + [_dp, _bp, _dp, _dp]
    L.or_map_lattice.restype = ctypes.c_int
    L.or_map_lattice.argtypes = [_ip, _dp, _dp, _fp, _fp, _fp]
    L.or_map_node_ray.restype = None
    L.or_map_node_ray.argtypes = [_fp, _fp, _ip, _fp]
    L.or_map_cell_of.restype = ctypes.c_int
    L.or_map_cell_of.argtypes = [_ip, _fp, _fp, _fp, _ip]
    L.or_map_cell_ids.restype = ctypes.c_long
    L.or_map_cell_ids.argtypes = [_ip, _fp, _fp, ctypes.c_long] + [_fp] * 6 + [_lp]
    L.or_map_trace_nodes.restype = ctypes.c_long
    L.or_map_trace_nodes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _fp, _fp,
                                     _dp, _bp]
    L.or_map_classify_cell.restype = ctypes.c_int
    L.or_map_classify_cell.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _fp, _fp,
                                       _ip, _dp, _bp, ctypes.c_long] + [_fp] * 6 + \
        [ctypes.c_double, _dp, _lp, _lp]
    L.or_map_build.restype = ctypes.c_long
    L.or_map_build.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _fp, _fp, _fp,
                               ctypes.c_long] + [_fp] * 6 + [ctypes.c_double, _dp, _bp, _bp, _dp]
    L.or_map_query.restype = ctypes.c_long
    L.or_map_query.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _fp, _fp, _fp,
                               _dp, _bp, _bp, ctypes.c_long] + [_fp] * 6 + [_dp, _bp]
    L.or_map_query_one.restype = ctypes.c_int
    L.or_map_query_one.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _fp, _fp, _fp,
                                   _fp, ctypes.c_long] + [_fp] * 6 + [ctypes.c_double, _dp, _ip]
    L.or_map_node_rays.restype = None
    L.or_map_node_rays.argtypes = [_ip, _fp, _fp] + [_fp] * 6
    L.or_map_interpolate.restype = None
    L.or_map_interpolate.argtypes = [_ip, _fp, _fp, _fp, _dp, _fp, _dp, _ip]


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


class Lens:
    """The oracle's own lens, built from a workloads.Prescription."""

    def __init__(self, presc):
        L = lib()
        self._buf = ctypes.create_string_buffer(L.or_lens_sizeof())
        S = presc.n_surfaces
        curv = np.array([s.curvature for s in presc.surfaces], np.float64)
        thick = np.array([s.thickness for s in presc.surfaces], np.float64)
        ap = np.array([s.aperture_r for s in presc.surfaces], np.float64)
        ga = np.array([s.glass_after for s in presc.surfaces], np.int32)
        ng = len(presc.glasses)
        gk = np.array([g.kind for g in presc.glasses] or [0], np.int32)
        gc = np.zeros((max(ng, 1), 8), np.float64)
        for i, g in enumerate(presc.glasses):
            gc[i, 0] = g.A
            gc[i, 1] = g.B
            gc[i, 2:5] = g.B3
            gc[i, 5:8] = g.C3
        rc = L.or_lens_init(self._buf, S, _ptr(curv, _dp), _ptr(thick, _dp), _ptr(ap, _dp),
                            _ptr(ga, _ip), ng, _ptr(gk, _ip), _ptr(gc, _dp),
                            presc.entrance_gap, presc.stop_after, presc.stop_offset, presc.stop_r,
                            presc.image_mode, presc.image_z, presc.lambda_ref_nm)
        if rc != 0:
            raise ValueError("oracle: bad prescription (or back focal distance <= 0)")
        for k, s in enumerate(presc.surfaces):
            kappa = float(getattr(s, "conic", 0.0))
            a = np.array(list(getattr(s, "asph", (0.0, 0.0, 0.0, 0.0))), np.float64)
            on = 1 if (kappa != 0.0 or np.any(a != 0.0) or getattr(s, "force_asphere", False)) else 0
            if on and L.or_lens_set_asphere(self._buf, k + 1, on, kappa, _ptr(a, _dp)) != 0:
                raise ValueError(f"oracle: asphere {k + 1}: aperture beyond the conic's domain")
        self.S = S
        self.presc = presc

    @property
    def handle(self):
        return self._buf

    def index(self, medium: int, lam_nm: float) -> float:
        return lib().or_index(self._buf, medium, lam_nm)

    def paraxial(self, lam_nm: float) -> Tuple[float, float]:
        efl = ctypes.c_double()
        bfd = ctypes.c_double()
        if lib().or_paraxial(self._buf, lam_nm, ctypes.byref(efl), ctypes.byref(bfd)) != 0:
            raise ValueError("afocal system")
        return efl.value, bfd.value

    def z_image(self) -> float:
        return lib().or_lens_get(self._buf, 0)

    def z_stop(self) -> float:
        return lib().or_lens_get(self._buf, 1)

    def vertex_z(self, k: int) -> float:
        return lib().or_lens_get(self._buf, 100 + k)

    def trace(self, rays, path: Tuple[int, int] = (0, 0)):
        """Trace FP32 rays in FP64.  Returns (out[n,6], valid[n] uint8 (bit3 bad input),
        edge[n], kmin[n])."""
        n = len(rays)
        arrs = [_f32(a) for a in rays.arrays()]
        out = np.zeros((n, 6), np.float64)
        valid = np.zeros(n, np.uint8)
        edge = np.zeros(n, np.float64)
        kmin = np.zeros(n, np.float64)
        lib().or_trace(self._buf, path[0], path[1], n, *[_ptr(a, _fp) for a in arrs],
                       _ptr(out, _dp), _ptr(valid, _bp), _ptr(edge, _dp), _ptr(kmin, _dp))
        return out, valid, edge, kmin

    def trace_states(self, x, y, dx, dy, dz, lam, path=(0, 0)):
        """(valid, out[6], states[m, 7]) with the state after each interaction."""
        out = np.zeros(6, np.float64)
        st = np.zeros((3 * 64 + 8, 7), np.float64)
        m = ctypes.c_int()
        v = lib().or_trace_states(self._buf, path[0], path[1], float(x), float(y), float(dx),
                                  float(dy), float(dz), float(lam), _ptr(out, _dp), _ptr(st, _dp),
                                  ctypes.byref(m))
        return v, out, st[:m.value].copy()

    def trace_one(self, x, y, dx, dy, dz, lam, path=(0, 0)):
        out = np.zeros(6, np.float64)
        e = ctypes.c_double()
        k = ctypes.c_double()
        v = lib().or_trace_one(self._buf, path[0], path[1], float(x), float(y), float(dx),
                               float(dy), float(dz), float(lam), _ptr(out, _dp), ctypes.byref(e),
                               ctypes.byref(k))
        return v, out, e.value, k.value


def fresnel(n1: float, n2: float, cos_i: float):
    """(tir, Rs, Rp, cos_t) at one interface."""
    Rs = ctypes.c_double()
    Rp = ctypes.c_double()
    ct = ctypes.c_double()
    tir = lib().or_fresnel(n1, n2, cos_i, ctypes.byref(Rs), ctypes.byref(Rp), ctypes.byref(ct))
    return bool(tir), Rs.value, Rp.value, ct.value


def path_sequence(S: int, i: int, j: int):
    n = 3 * 64 + 4
    surf = (ctypes.c_int * n)()
    typ = (ctypes.c_int * n)()
    d = (ctypes.c_int * n)()
    K = lib().or_path_sequence(S, i, j, surf, typ, d)
    if K < 0:
        raise ValueError("bad path")
    return list(surf[:K]), list(typ[:K]), list(d[:K])


def path_code(S: int, i: int, j: int) -> int:
    return int(lib().or_path_code(S, i, j))


def path_ij(S: int, pid: int) -> Tuple[int, int]:
    i = ctypes.c_int()
    j = ctypes.c_int()
    if lib().or_path_ij(S, pid, ctypes.byref(i), ctypes.byref(j)) != 0:
        raise ValueError("bad path id")
    return i.value, j.value


# ------------------------------------------------------------------------------------------
# tabulated map
# ------------------------------------------------------------------------------------------

class Lattice:
    """FP32 lattice constants over the 5-D box (x, y, s_x, s_y, lambda)."""

    def __init__(self, res, lo, hi):
        self.res = np.ascontiguousarray(res, np.int32)
        lo = np.ascontiguousarray(lo, np.float64)
        hi = np.ascontiguousarray(hi, np.float64)
        self.lo_f = np.zeros(5, np.float32)
        self.step_f = np.zeros(5, np.float32)
        self.inv_f = np.zeros(5, np.float32)
        if lib().or_map_lattice(_ptr(self.res, _ip), _ptr(lo, _dp), _ptr(hi, _dp),
                                _ptr(self.lo_f, _fp), _ptr(self.step_f, _fp),
                                _ptr(self.inv_f, _fp)) != 0:
            raise ValueError("bad lattice")

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.res.astype(np.int64)))

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.res.astype(np.int64) - 1))

    def args(self):
        return (_ptr(self.res, _ip), _ptr(self.lo_f, _fp), _ptr(self.step_f, _fp),
                _ptr(self.inv_f, _fp))

    def node_ray(self, idx) -> np.ndarray:
        idx = np.ascontiguousarray(idx, np.int32)
        ray = np.zeros(6, np.float32)
        lib().or_map_node_ray(_ptr(self.lo_f, _fp), _ptr(self.step_f, _fp), _ptr(idx, _ip),
                              _ptr(ray, _fp))
        return ray

    def node_rays(self):
        """Entrance rays of every lattice node, in table order (a workloads.Rays)."""
        from paper_2605_04017_gb300.workloads import Rays
        N = self.n_nodes
        arrs = [np.zeros(N, np.float32) for _ in range(6)]
        lib().or_map_node_rays(_ptr(self.res, _ip), _ptr(self.lo_f, _fp), _ptr(self.step_f, _fp),
                               *[_ptr(a, _fp) for a in arrs])
        return Rays(*arrs)

    def cell_ids(self, rays) -> np.ndarray:
        n = len(rays)
        arrs = [_f32(a) for a in rays.arrays()]
        out = np.zeros(n, np.int64)
        lib().or_map_cell_ids(_ptr(self.res, _ip), _ptr(self.lo_f, _fp), _ptr(self.inv_f, _fp), n,
                              *[_ptr(a, _fp) for a in arrs], out.ctypes.data_as(_lp))
        return out

    def cell_of(self, ray6) -> Optional[np.ndarray]:
        ray6 = _f32(ray6)
        cell = np.zeros(5, np.int32)
        ok = lib().or_map_cell_of(_ptr(self.res, _ip), _ptr(self.lo_f, _fp), _ptr(self.inv_f, _fp),
                                  _ptr(ray6, _fp), _ptr(cell, _ip))
        return cell if ok else None

    def interpolate(self, corner6: np.ndarray, ray6) -> Tuple[np.ndarray, np.ndarray]:
        corner6 = np.ascontiguousarray(corner6, np.float64)
        ray6 = _f32(ray6)
        out = np.zeros(6, np.float64)
        cell = np.zeros(5, np.int32)
        r, lo, st, inv = self.args()
        lib().or_map_interpolate(r, lo, st, inv, _ptr(corner6, _dp), _ptr(ray6, _fp),
                                 _ptr(out, _dp), _ptr(cell, _ip))
        return out, cell


class TableMap:
    """The oracle's own tabulated map of one path, built from scratch."""

    def __init__(self, lens: Lens, path: Tuple[int, int], lattice: Lattice, fit_rays,
                 tol: float = float("inf")):
        self.lens, self.path, self.lat, self.tol = lens, path, lattice, tol
        N, NC = lattice.n_nodes, lattice.n_cells
        self.node6 = np.zeros((N, 6), np.float64)
        self.node_valid = np.zeros(N, np.uint8)
        self.cell_class = np.zeros(NC, np.uint8)
        self.cell_maxres = np.zeros(NC, np.float64)
        arrs = [_f32(a) for a in fit_rays.arrays()]
        r, lo, st, inv = lattice.args()
        lib().or_map_build(lens.handle, path[0], path[1], r, lo, st, inv, len(fit_rays),
                           *[_ptr(a, _fp) for a in arrs], tol, _ptr(self.node6, _dp),
                           _ptr(self.node_valid, _bp), _ptr(self.cell_class, _bp),
                           _ptr(self.cell_maxres, _dp))

    def quantize16(self):
        """Replace the node values by their 16-bit decoded form (quantize16);
        returns the six steps."""
        self.node6, steps = quantize16(self.node6, self.node_valid)
        return steps

    def query(self, rays):
        n = len(rays)
        arrs = [_f32(a) for a in rays.arrays()]
        out = np.zeros((n, 6), np.float64)
        flags = np.zeros(n, np.uint8)
        r, lo, st, inv = self.lat.args()
        lib().or_map_query(self.lens.handle, self.path[0], self.path[1], r, lo, st, inv,
                           _ptr(self.node6, _dp), _ptr(self.node_valid, _bp),
                           _ptr(self.cell_class, _bp), n, *[_ptr(a, _fp) for a in arrs],
                           _ptr(out, _dp), _ptr(flags, _bp))
        return out, flags


def quantize16(node6: np.ndarray, node_valid: np.ndarray):
    """The half-size node table (16 bits per output): output k of a node is
    stored as an integer q in [-32768, 32767] times step_k = 2^(e_k - 15),
    where 2^e_k is the smallest power of two above the largest |value| of
    output k over the valid nodes (step 2^-15 if there is none), and
    q = value / step_k rounded to the nearest integer, ties to even;
    invalid nodes store 0.  Returns the decoded node values (q * step, FP64)
    and the six steps.  A power-of-two step makes value / step exact, so the
    only rounding is the one to an integer."""
    v = np.asarray(node6, np.float64)
    ok = np.asarray(node_valid) != 0
    steps = np.empty(6, np.float64)
    out = np.zeros_like(v)
    for k in range(6):
        m = float(np.abs(v[ok, k]).max()) if ok.any() else 0.0
        e = math.frexp(m)[1] if m > 0.0 else 0      # 2^(e-1) <= m < 2^e
        steps[k] = math.ldexp(1.0, e - 15)
        q = np.clip(np.rint(v[:, k] / steps[k]), -32768, 32767)
        out[:, k] = np.where(ok, q * steps[k], 0.0)
    return out, steps


def trace_nodes(lens: Lens, path, lattice: Lattice):
    N = lattice.n_nodes
    node6 = np.zeros((N, 6), np.float64)
    valid = np.zeros(N, np.uint8)
    r, lo, st, inv = lattice.args()
    lib().or_map_trace_nodes(lens.handle, path[0], path[1], r, lo, st, _ptr(node6, _dp),
                             _ptr(valid, _bp))
    return node6, valid


def classify_cell(lens: Lens, path, lattice: Lattice, cell, fit_rays, tol=float("inf")):
    """Class of one cell from its 32 freshly traced corners and the given fit rays
    (which the caller selects as the rays inside the cell)."""
    cell = np.ascontiguousarray(cell, np.int32)
    corner6 = np.zeros((32, 6), np.float64)
    cv = np.zeros(32, np.uint8)
    for k in range(32):
        idx = np.array([cell[d] + ((k >> (4 - d)) & 1) for d in range(5)], np.int32)
        ray = lattice.node_ray(idx)
        v, out, _, _ = lens.trace_one(*ray, path=path)
        corner6[k] = out
        cv[k] = 1 if v == 1 else 0
    arrs = [_f32(a) for a in fit_rays.arrays()]
    mr = ctypes.c_double()
    nv = ctypes.c_long()
    ni = ctypes.c_long()
    r, lo, st, inv = lattice.args()
    cls = lib().or_map_classify_cell(lens.handle, path[0], path[1], r, lo, st, _ptr(cell, _ip),
                                     _ptr(corner6, _dp), _ptr(cv, _bp), len(fit_rays),
                                     *[_ptr(a, _fp) for a in arrs], tol, ctypes.byref(mr),
                                     ctypes.byref(nv), ctypes.byref(ni))
    return cls, corner6, cv, mr.value
