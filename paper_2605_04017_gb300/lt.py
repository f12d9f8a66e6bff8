"""Thin ctypes binding of liblt.so (the C ABI in include/lt.h).

Argument marshalling only: every step of the lens-transport path runs in
the library's CUDA kernels.  PyTorch tensors serve as device memory and
their streams as cudaStream_t; nothing here computes optics.  If the
library has not been built, importing works but every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import build as _build

LT_OK = 0
LT_EINVAL = -1
LT_ENOMEM = -2
LT_ECUDA = -3
LT_EBUSY = -4
LT_ETIMEOUT = -5
LT_ENOTREADY = -6
LT_EBADLENS = -7
LT_EIO = -8

FLAG_VALID = 0x01
FLAG_NEAR_EDGE = 0x02
FLAG_NEAR_TIR = 0x04
FLAG_BAD_INPUT = 0x08
FLAG_TRACED = 0x10
FLAG_OUTSIDE = 0x20
FLAG_GRAZING = 0x40

MAX_SURFACES = 32
MAX_GLASSES = 32


class LTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lt error {code}: {msg}")
        self.code = code


class c_glass(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("A", ctypes.c_double), ("B", ctypes.c_double),
                ("B3", ctypes.c_double * 3), ("C3", ctypes.c_double * 3)]


class c_surface(ctypes.Structure):
    _fields_ = [("curvature", ctypes.c_double), ("thickness", ctypes.c_double),
                ("aperture_r", ctypes.c_double), ("glass_after", ctypes.c_int),
                ("conic", ctypes.c_double), ("asph", ctypes.c_double * 4)]


class c_prescription(ctypes.Structure):
    _fields_ = [("n_surfaces", ctypes.c_int), ("surfaces", ctypes.POINTER(c_surface)),
                ("n_glasses", ctypes.c_int), ("glasses", ctypes.POINTER(c_glass)),
                ("entrance_gap", ctypes.c_double), ("stop_after", ctypes.c_int),
                ("stop_offset", ctypes.c_double), ("stop_r", ctypes.c_double),
                ("image_mode", ctypes.c_int), ("image_z", ctypes.c_double),
                ("lambda_ref_nm", ctypes.c_double), ("edge_eps_mm", ctypes.c_double),
                ("grazing_k", ctypes.c_double)]


_fptr = ctypes.c_void_p


class c_rays_in(ctypes.Structure):
    _fields_ = [("x", _fptr), ("y", _fptr), ("dx", _fptr), ("dy", _fptr), ("dz", _fptr)]


class c_rays_out(ctypes.Structure):
    _fields_ = [("x", _fptr), ("y", _fptr), ("dx", _fptr), ("dy", _fptr), ("dz", _fptr),
                ("I", _fptr), ("flags", _fptr)]


_LIB: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded liblt.so.  Raises if it has not been built: there is no
    fallback implementation."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"liblt.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        _declare(L)
        _LIB = L
    return _LIB


def _declare(L: ctypes.CDLL) -> None:
    vp = ctypes.c_void_p
    st = ctypes.c_int
    L.lt_last_error.restype = ctypes.c_char_p
    L.lt_version.restype = ctypes.c_char_p
    L.lt_create_lens.restype = st
    L.lt_create_lens.argtypes = [ctypes.POINTER(c_prescription), ctypes.POINTER(vp)]
    L.lt_destroy_lens.restype = None
    L.lt_destroy_lens.argtypes = [vp]
    L.lt_lens_paraxial.restype = st
    L.lt_lens_paraxial.argtypes = [vp, ctypes.c_double] + [ctypes.POINTER(ctypes.c_double)] * 3
    L.lt_lens_n_paths.restype = ctypes.c_int32
    L.lt_lens_n_paths.argtypes = [vp]
    L.lt_path_ij.restype = st
    L.lt_path_ij.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_int32)]
    L.lt_path_id.restype = ctypes.c_int32
    L.lt_path_id.argtypes = [ctypes.c_int32] * 3
    L.lt_path_code.restype = ctypes.c_uint64
    L.lt_path_code.argtypes = [ctypes.c_int32] * 3
    L.lt_trace.restype = st
    L.lt_trace.argtypes = [vp, ctypes.POINTER(c_rays_in), vp, ctypes.c_int32,
                           ctypes.POINTER(c_rays_out), ctypes.c_size_t, vp]
    L.lt_trace_host.restype = st
    L.lt_trace_host.argtypes = [vp, ctypes.POINTER(c_rays_in), vp, ctypes.c_int32,
                                ctypes.POINTER(c_rays_out), ctypes.c_size_t]
    L.lt_tracer_math.restype = st
    L.lt_tracer_math.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]


def check(code: int) -> None:
    if code != LT_OK:
        raise LTError(code, lib().lt_last_error().decode())


def last_error() -> str:
    return lib().lt_last_error().decode()


def version() -> str:
    return lib().lt_version().decode()


def path_id(S: int, i: int, j: int) -> int:
    return int(lib().lt_path_id(S, i, j))


def path_ij(S: int, pid: int):
    i = ctypes.c_int32()
    j = ctypes.c_int32()
    check(lib().lt_path_ij(S, pid, ctypes.byref(i), ctypes.byref(j)))
    return i.value, j.value


def path_code(S: int, i: int, j: int) -> int:
    return int(lib().lt_path_code(S, i, j))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    return int(t)


class Lens:
    """A lens resident in the library, created from a workloads.Prescription
    (or anything with the same attributes)."""

    def __init__(self, presc, edge_eps_mm: float = 0.0, grazing_k: float = 0.0):
        S = len(presc.surfaces)
        self._surfs = (c_surface * max(S, 1))()
        for k, s in enumerate(presc.surfaces):
            self._surfs[k] = c_surface(s.curvature, s.thickness, s.aperture_r, s.glass_after,
                                       float(getattr(s, "conic", 0.0)),
                                       (ctypes.c_double * 4)(*getattr(s, "asph", (0.0, 0.0, 0.0, 0.0))))
        ng = len(presc.glasses)
        self._glasses = (c_glass * max(ng, 1))()
        for g, G in enumerate(presc.glasses):
            self._glasses[g] = c_glass(G.kind, G.A, G.B, (ctypes.c_double * 3)(*G.B3),
                                       (ctypes.c_double * 3)(*G.C3))
        self._p = c_prescription(S, self._surfs, ng, self._glasses, presc.entrance_gap,
                                 presc.stop_after, presc.stop_offset, presc.stop_r,
                                 presc.image_mode, presc.image_z, presc.lambda_ref_nm, edge_eps_mm,
                                 grazing_k)
        h = ctypes.c_void_p()
        check(lib().lt_create_lens(ctypes.byref(self._p), ctypes.byref(h)))
        self.handle = h
        self.S = S
        self.presc = presc

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().lt_destroy_lens(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_paths(self) -> int:
        return int(lib().lt_lens_n_paths(self.handle))

    def reversed(self, sensor_z: float, out_z: float) -> "Lens":
        """lt_reverse_lens: this lens seen from its image side (backward path
        tracing), entrance plane at the forward plane z = sensor_z, image
        plane at the forward plane z = out_z."""
        L = lib()
        L.lt_reverse_lens.restype = ctypes.c_int
        L.lt_reverse_lens.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        h = ctypes.c_void_p()
        check(L.lt_reverse_lens(self.handle, sensor_z, out_z, ctypes.byref(h)))
        r = Lens.__new__(Lens)
        r.handle = h
        r.S = self.S
        r.presc = None
        return r

    def paraxial(self, lam_nm: float):
        e, b, z = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().lt_lens_paraxial(self.handle, lam_nm, ctypes.byref(e), ctypes.byref(b),
                                     ctypes.byref(z)))
        return e.value, b.value, z.value


def rays_in(x, y, dx, dy, dz) -> c_rays_in:
    return c_rays_in(_ptr(x), _ptr(y), _ptr(dx), _ptr(dy), _ptr(dz))


def rays_out(x, y, dx, dy, dz, I, flags) -> c_rays_out:
    return c_rays_out(_ptr(x), _ptr(y), _ptr(dx), _ptr(dy), _ptr(dz), _ptr(I), _ptr(flags))


def trace(lens: Lens, inp: Sequence, lam, path_id: int, out: Sequence, n: int, stream=None):
    """lt_trace on device tensors: inp = (x, y, dx, dy, dz), out = (x, y, dx, dy, dz, I, flags)."""
    ri = rays_in(*inp)
    ro = rays_out(*out)
    check(lib().lt_trace(lens.handle, ctypes.byref(ri), _ptr(lam), path_id, ctypes.byref(ro), n,
                         _stream_handle(stream)))


def tracer_math(x, rcp, sqrt_out, n: int, stream=None):
    """lt_tracer_math on device float tensors: the tracer's reciprocal and
    square root of each x[i]."""
    check(lib().lt_tracer_math(_ptr(x), _ptr(rcp), _ptr(sqrt_out), n, _stream_handle(stream)))


def trace_host(lens: Lens, inp: Sequence, lam, path_id: int, out: Sequence, n: int):
    """lt_trace_host on host arrays (numpy or pinned CPU tensors)."""
    ri = rays_in(*inp)
    ro = rays_out(*out)
    check(lib().lt_trace_host(lens.handle, ctypes.byref(ri), _ptr(lam), path_id, ctypes.byref(ro),
                              n))


class c_paths_out(ctypes.Structure):
    _fields_ = [("x", _fptr), ("y", _fptr), ("dx", _fptr), ("dy", _fptr), ("dz", _fptr),
                ("I", _fptr), ("flags", ctypes.c_void_p), ("ray_index", ctypes.c_void_p),
                ("valid_count", ctypes.c_void_p), ("capacity", ctypes.c_size_t)]


def _declare_paths(L: ctypes.CDLL) -> None:
    L.lt_trace_paths.restype = ctypes.c_int
    L.lt_trace_paths.argtypes = [ctypes.c_void_p, ctypes.POINTER(c_rays_in), ctypes.c_void_p,
                                 ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.POINTER(c_paths_out), ctypes.c_size_t, ctypes.c_void_p]


def trace_paths(lens: Lens, inp: Sequence, lam, lam_stride: int, path_ids, out, n: int,
                stream=None) -> None:
    """lt_trace_paths on device tensors.  out: a batch.PathsOut (or any object
    with f = [x, y, dx, dy, dz, I], flags, ray_index, valid_count, capacity)."""
    import numpy as np
    ids = np.ascontiguousarray(path_ids, np.int32)
    ri = rays_in(*inp)
    po = c_paths_out(*[_ptr(t) for t in out.f], _ptr(out.flags), _ptr(out.ray_index),
                     _ptr(out.valid_count), out.capacity)
    check(lib().lt_trace_paths(lens.handle, ctypes.byref(ri), _ptr(lam), lam_stride,
                               ids.ctypes.data, len(ids), ctypes.byref(po), n,
                               _stream_handle(stream)))


class c_sensor(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pixel_mm", ctypes.c_double),
                ("weight", ctypes.c_float), ("per_path", ctypes.c_int32)]


def splat_paths(lens: Lens, inp: Sequence, lam, lam_stride: int, path_ids, n: int, width: int,
                height: int, pixel_mm: float, image, weight: float = 1.0, per_path: bool = False,
                stream=None) -> None:
    """lt_splat_paths: forward light tracing of n rays along the given paths
    onto a sensor image (device float tensor [n_images, height, width],
    accumulated into)."""
    import numpy as np
    L = lib()
    L.lt_splat_paths.restype = ctypes.c_int
    L.lt_splat_paths.argtypes = [ctypes.c_void_p, ctypes.POINTER(c_rays_in), ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(c_sensor),
                                 ctypes.c_void_p, ctypes.c_void_p]
    ids = np.ascontiguousarray(path_ids, np.int32)
    ri = rays_in(*inp)
    sen = c_sensor(width, height, pixel_mm, weight, 1 if per_path else 0)
    check(L.lt_splat_paths(lens.handle, ctypes.byref(ri), _ptr(lam), lam_stride, ids.ctypes.data, len(ids), n,
                           ctypes.byref(sen), _ptr(image), _stream_handle(stream)))


class c_mcmc_opts(ctypes.Structure):
    _fields_ = [("path_id", ctypes.c_int32), ("lo", ctypes.c_double * 5), ("hi", ctypes.c_double * 5),
                ("seed", ctypes.c_uint64), ("chains", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("small", ctypes.c_double), ("p_large", ctypes.c_double), ("init_tries", ctypes.c_int32)]


class c_samples_out(ctypes.Structure):
    _fields_ = [("x", _fptr), ("y", _fptr), ("dx", _fptr), ("dy", _fptr), ("dz", _fptr),
                ("lambda_nm", _fptr), ("flags", ctypes.c_void_p), ("accepted", ctypes.c_void_p)]


def mcmc_sample(lens: Lens, path_id: int, lo, hi, seed: int, chains: int, steps: int, small: float,
                p_large: float, init_tries: int, stream=None):
    """lt_mcmc_sample: returns (device tensors [x, y, dx, dy, dz, lambda] of
    chains * steps samples, flags, accepted per chain)."""
    import torch
    L = lib()
    L.lt_mcmc_sample.restype = ctypes.c_int
    L.lt_mcmc_sample.argtypes = [ctypes.c_void_p, ctypes.POINTER(c_mcmc_opts), ctypes.POINTER(c_samples_out),
                                 ctypes.c_void_p]
    n = chains * steps
    f = [torch.empty(max(n, 1), dtype=torch.float32, device="cuda") for _ in range(6)]
    flags = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    acc = torch.empty(max(chains, 1), dtype=torch.int32, device="cuda")
    o = c_mcmc_opts(path_id, (ctypes.c_double * 5)(*lo), (ctypes.c_double * 5)(*hi), seed, chains, steps,
                    small, p_large, init_tries)
    out = c_samples_out(*[_ptr(t) for t in f], _ptr(flags), _ptr(acc))
    check(L.lt_mcmc_sample(lens.handle, ctypes.byref(o), ctypes.byref(out), _stream_handle(stream)))
    return f, flags, acc


class FitRays:
    """A device training set for lt_mlp_train: inp = [x, y, dx, dy, dz], lam,
    n, and n_uniform (how many leading rays are uniform draws of the box)."""

    def __init__(self, inp, lam, n_uniform=0):
        self.inp, self.lam, self.n = list(inp), lam, int(lam.numel())
        self.n_uniform = int(n_uniform)


def valid_region_fit(lens: Lens, path_id: int, lo, hi, uniform, chains: int, steps: int, seed: int,
                     small: float = 0.03, p_large: float = 0.05, init_tries: int = 64, stream=None) -> FitRays:
    """Training rays of one path as Sec. 5.1 collects them: the regressor
    wants rays spread over the path's valid region, which uniform draws of
    the input box seldom hit on a ghost path, so a Markov chain sampler whose
    target is the path's binary visibility (lt_mcmc_sample) supplies them;
    the classifier wants valid and invalid rays in about equal numbers, which
    the uniform draws (mostly invalid on a sparse path) complete.  Returns
    `uniform` (a batch.DeviceRays) followed by the states of every chain that
    started (chains x steps samples at most), with n_uniform set so that
    lt_mlp_train corrects its classifier for the sampler's extra valid rays.
    Joining the two sets is a device copy; tracing, labels and training are
    the library's."""
    import torch
    f, flags, _ = mcmc_sample(lens, path_id, lo, hi, seed, chains, steps, small, p_large, init_tries, stream)
    torch.cuda.synchronize()          # the joins below run on torch's current stream
    m = chains * steps
    keep = flags[:m] != 0
    inp = [torch.cat([u, s[:m][keep]]) for u, s in zip(uniform.inp, f[:5])]
    lam = torch.cat([uniform.lam, f[5][:m][keep]])
    return FitRays(inp, lam, uniform.n)


# ------------------------------------------------------------------ maps

QUERY_TABLE = 0
QUERY_NO_MASK = 1

CELL_INVALID, CELL_VALID, CELL_BOUNDARY = 0, 1, 2


class c_map_opts(ctypes.Structure):
    _fields_ = [("path_id", ctypes.c_int32), ("res", ctypes.c_int32 * 5),
                ("lo", ctypes.c_double * 5), ("hi", ctypes.c_double * 5),
                ("max_residual_mm", ctypes.c_double),
                ("fit_x", _fptr), ("fit_y", _fptr), ("fit_dx", _fptr), ("fit_dy", _fptr),
                ("fit_dz", _fptr), ("fit_lambda", _fptr), ("n_fit", ctypes.c_size_t),
                ("node_format", ctypes.c_int32)]


NODE_F32, NODE_S16 = 0, 1


class c_map_stats(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint64), ("n_cells", ctypes.c_uint64),
                ("valid_nodes", ctypes.c_uint64), ("cells_invalid", ctypes.c_uint64),
                ("cells_valid", ctypes.c_uint64), ("cells_boundary", ctypes.c_uint64),
                ("fit_inside", ctypes.c_uint64), ("fit_valid", ctypes.c_uint64),
                ("fit_residual_rms_mm", ctypes.c_double), ("fit_residual_max_mm", ctypes.c_double),
                ("table_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_double),
                ("node_format", ctypes.c_int32), ("node_step", ctypes.c_float * 6)]


class c_poly_opts(ctypes.Structure):
    _fields_ = [("path_id", ctypes.c_int32), ("rho", ctypes.c_double), ("smax", ctypes.c_double),
                ("lam_lo", ctypes.c_double), ("lam_hi", ctypes.c_double), ("degree", ctypes.c_int32),
                ("patches", ctypes.c_int32 * 4), ("cells", ctypes.c_int32 * 4),
                ("samples", ctypes.c_int32), ("max_residual_mm", ctypes.c_double),
                ("fit_x", _fptr), ("fit_y", _fptr), ("fit_dx", _fptr), ("fit_dy", _fptr),
                ("fit_dz", _fptr), ("fit_lambda", _fptr), ("n_fit", ctypes.c_size_t)]


class c_poly_stats(ctypes.Structure):
    _fields_ = [("patches", ctypes.c_uint32), ("patches_fit", ctypes.c_uint32),
                ("terms", ctypes.c_uint32), ("samples_traced", ctypes.c_uint64),
                ("samples_valid", ctypes.c_uint64), ("sample_residual_max_mm", ctypes.c_double),
                ("corner_residual_max_mm", ctypes.c_double)]


POLY_MAX_DEGREE = 5


def _declare_maps(L: ctypes.CDLL) -> None:
    vp = ctypes.c_void_p
    st = ctypes.c_int
    L.lt_build_poly_map.restype = st
    L.lt_build_poly_map.argtypes = [vp, ctypes.POINTER(c_poly_opts), ctypes.POINTER(vp), vp]
    L.lt_poly_stats_get.restype = st
    L.lt_poly_stats_get.argtypes = [vp, ctypes.POINTER(c_poly_stats)]
    L.lt_poly_export.restype = st
    L.lt_poly_export.argtypes = [vp, vp, vp, vp]
    L.lt_build_map.restype = st
    L.lt_build_map.argtypes = [vp, ctypes.POINTER(c_map_opts), ctypes.POINTER(vp), vp]
    L.lt_destroy_map.restype = None
    L.lt_destroy_map.argtypes = [vp]
    L.lt_map_stats_get.restype = st
    L.lt_map_stats_get.argtypes = [vp, ctypes.POINTER(c_map_stats)]
    L.lt_query.restype = st
    L.lt_query.argtypes = [vp, ctypes.POINTER(c_rays_in), vp, ctypes.POINTER(c_rays_out),
                           ctypes.c_size_t, ctypes.c_int32, vp]
    L.lt_query_host.restype = st
    L.lt_query_host.argtypes = [vp, ctypes.POINTER(c_rays_in), vp, ctypes.POINTER(c_rays_out),
                                ctypes.c_size_t, ctypes.c_int32]
    L.lt_map_export.restype = st
    L.lt_map_export.argtypes = [vp, vp, vp, vp]
    L.lt_map_save.restype = st
    L.lt_map_save.argtypes = [vp, ctypes.c_char_p]
    L.lt_map_load.restype = st
    L.lt_map_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]


_old_declare = _declare


def _declare(L: ctypes.CDLL) -> None:  # noqa: F811
    _old_declare(L)
    _declare_maps(L)


class Map:
    """A map resident on the device (lt_build_map / lt_map_load)."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    @classmethod
    def build(cls, lens: Lens, path_id: int, res, lo, hi, fit=None, max_residual_mm: float = 0.0,
              stream=None, node_format: int = NODE_F32) -> "Map":
        """fit: a batch.DeviceRays (or None); node_format NODE_F32 or NODE_S16."""
        o = c_map_opts()
        o.path_id = path_id
        o.node_format = node_format
        for d in range(5):
            o.res[d] = int(res[d])
            o.lo[d] = float(lo[d])
            o.hi[d] = float(hi[d])
        o.max_residual_mm = max_residual_mm
        if fit is not None:
            o.fit_x, o.fit_y, o.fit_dx, o.fit_dy, o.fit_dz = [_ptr(t) for t in fit.inp]
            o.fit_lambda = _ptr(fit.lam)
            o.n_fit = fit.n
        h = ctypes.c_void_p()
        check(lib().lt_build_map(lens.handle, ctypes.byref(o), ctypes.byref(h),
                                 _stream_handle(stream)))
        return cls(h)

    @classmethod
    def build_poly(cls, lens: Lens, path_id: int, rho: float, smax: float, degree: int, patches,
                   cells, samples: int, lam_lo: float = 380.0, lam_hi: float = 780.0, fit=None,
                   max_residual_mm: float = 0.0, stream=None) -> "Map":
        """lt_build_poly_map; fit: a batch.DeviceRays (or None)."""
        o = c_poly_opts()
        o.path_id = path_id
        o.rho, o.smax, o.lam_lo, o.lam_hi = float(rho), float(smax), float(lam_lo), float(lam_hi)
        o.degree = int(degree)
        for k in range(4):
            o.patches[k] = int(patches[k])
            o.cells[k] = int(cells[k])
        o.samples = int(samples)
        o.max_residual_mm = float(max_residual_mm)
        if fit is not None:
            o.fit_x, o.fit_y, o.fit_dx, o.fit_dy, o.fit_dz = [_ptr(t) for t in fit.inp]
            o.fit_lambda = _ptr(fit.lam)
            o.n_fit = fit.n
        h = ctypes.c_void_p()
        check(lib().lt_build_poly_map(lens.handle, ctypes.byref(o), ctypes.byref(h),
                                      _stream_handle(stream)))
        return cls(h)

    def poly_stats(self) -> dict:
        s = c_poly_stats()
        check(lib().lt_poly_stats_get(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in c_poly_stats._fields_}

    def poly_export(self):
        """(coef [patches, terms, 5] FP64, exps [terms, 4], patch_ok [patches])."""
        import numpy as np
        ps = self.poly_stats()
        P, T = ps["patches"], ps["terms"]
        coef = np.empty((P, T, 5), np.float64)
        exps = np.empty((T, 4), np.int32)
        ok = np.empty(P, np.uint8)
        check(lib().lt_poly_export(self.handle, coef.ctypes.data, exps.ctypes.data, ok.ctypes.data))
        return coef, exps, ok

    def export_mask(self, n_nodes: int, n_cells: int):
        """(node_valid [n_nodes], cell_class [n_cells]) of either kind of map."""
        import numpy as np
        nv = np.empty(n_nodes, np.uint8)
        cc = np.empty(n_cells, np.uint8)
        check(lib().lt_map_export(self.handle, None, nv.ctypes.data, cc.ctypes.data))
        return nv, cc

    @classmethod
    def load(cls, path: str) -> "Map":
        h = ctypes.c_void_p()
        check(lib().lt_map_load(path.encode(), ctypes.byref(h)))
        return cls(h)

    def save(self, path: str) -> None:
        check(lib().lt_map_save(self.handle, path.encode()))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().lt_destroy_map(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = c_map_stats()
        check(lib().lt_map_stats_get(self.handle, ctypes.byref(s)))
        return {k: (list(getattr(s, k)) if isinstance(getattr(s, k), ctypes.Array) else getattr(s, k))
                for k, _ in c_map_stats._fields_}

    def query(self, inp: Sequence, lam, out: Sequence, n: int, mode: int = QUERY_TABLE,
              stream=None) -> None:
        ri = rays_in(*inp)
        ro = rays_out(*out)
        check(lib().lt_query(self.handle, ctypes.byref(ri), _ptr(lam), ctypes.byref(ro), n, mode,
                             _stream_handle(stream)))

    def query_host(self, inp: Sequence, lam, out: Sequence, n: int, mode: int = QUERY_TABLE):
        ri = rays_in(*inp)
        ro = rays_out(*out)
        check(lib().lt_query_host(self.handle, ctypes.byref(ri), _ptr(lam), ctypes.byref(ro), n,
                                  mode))

    def export(self, n_nodes: int, n_cells: int):
        import numpy as np
        node6 = np.empty((n_nodes, 6), np.float32)
        nv = np.empty(n_nodes, np.uint8)
        cc = np.empty(n_cells, np.uint8)
        check(lib().lt_map_export(self.handle, node6.ctypes.data, nv.ctypes.data, cc.ctypes.data))
        return node6, nv, cc


# ------------------------------------------------------------------ profiling

class c_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("work", ctypes.c_int64)]


def profile_enable(on: bool = True) -> None:
    L = lib()
    L.lt_profile_enable.restype = ctypes.c_int
    L.lt_profile_enable.argtypes = [ctypes.c_int32]
    check(L.lt_profile_enable(1 if on else 0))


def profile_read(reset: bool = True) -> dict:
    """{kernel name: (launches, total device ms, work units)} since the last reset."""
    L = lib()
    L.lt_profile_read.restype = ctypes.c_int
    L.lt_profile_read.argtypes = [ctypes.POINTER(c_kernel_time), ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
    buf = (c_kernel_time * 64)()
    n = ctypes.c_int32()
    check(L.lt_profile_read(buf, 64, ctypes.byref(n), 1 if reset else 0))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), int(buf[i].work))
            for i in range(min(n.value, 64))}


# ------------------------------------------------------------------ allocation-free query

NOALLOC_MAX_RAYS = 1 << 19


def query_noalloc(gmap: "Map", inp: Sequence, lam, out: Sequence, n: int,
                  mode: int = QUERY_TABLE, stream=None) -> None:
    """lt_query_noalloc: the map query under an allocation-free contract
    (n <= NOALLOC_MAX_RAYS = 2^19)."""
    L = lib()
    L.lt_query_noalloc.restype = ctypes.c_int
    L.lt_query_noalloc.argtypes = [ctypes.c_void_p, ctypes.POINTER(c_rays_in), ctypes.c_void_p,
                                   ctypes.POINTER(c_rays_out), ctypes.c_size_t, ctypes.c_int32,
                                   ctypes.c_void_p]
    ri = rays_in(*inp)
    ro = rays_out(*out)
    check(L.lt_query_noalloc(gmap.handle, ctypes.byref(ri), _ptr(lam), ctypes.byref(ro), n, mode,
                             _stream_handle(stream)))


# ------------------------------------------------------------------ learned maps

MLP_REG_PARAMS = 4582
MLP_CLS_PARAMS = 1249
MLP_F32, MLP_BF16, MLP_F16, MLP_F32_NOCLS = 0, 1, 2, 3


class c_mlp_frame(ctypes.Structure):
    _fields_ = [("path_id", ctypes.c_int32), ("rho", ctypes.c_double), ("wmax", ctypes.c_double),
                ("lam_lo", ctypes.c_double), ("lam_hi", ctypes.c_double)]


class c_mlp_opts(ctypes.Structure):
    _fields_ = [("frame", c_mlp_frame),
                ("fit_x", _fptr), ("fit_y", _fptr), ("fit_dx", _fptr), ("fit_dy", _fptr),
                ("fit_dz", _fptr), ("fit_lambda", _fptr), ("n_fit", ctypes.c_size_t),
                ("init_reg", _fptr), ("init_cls", _fptr),
                ("reg_steps", ctypes.c_int32), ("reg_batch", ctypes.c_int32),
                ("cls_steps", ctypes.c_int32), ("cls_batch", ctypes.c_int32),
                ("lr", ctypes.c_double), ("lr_decay", ctypes.c_double),
                ("decay_every", ctypes.c_int32),
                ("ft_steps", ctypes.c_int32), ("ft_batch", ctypes.c_int32), ("ft_lr", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("n_fit_uniform", ctypes.c_uint64)]


class c_mlp_stats(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_uint64), ("n_valid", ctypes.c_uint64),
                ("reg_loss", ctypes.c_double), ("cls_loss", ctypes.c_double),
                ("t_mean", ctypes.c_double * 6), ("t_std", ctypes.c_double * 6),
                ("train_ms", ctypes.c_double), ("tc_wait_timeouts", ctypes.c_uint64),
                ("n_valid_uniform", ctypes.c_uint64), ("cls_prior_shift", ctypes.c_double)]


def _declare_mlp(L: ctypes.CDLL) -> None:
    vp = ctypes.c_void_p
    st = ctypes.c_int
    L.lt_mlp_train.restype = st
    L.lt_mlp_train.argtypes = [vp, ctypes.POINTER(c_mlp_opts), ctypes.POINTER(vp), vp]
    L.lt_mlp_create.restype = st
    L.lt_mlp_create.argtypes = [vp, ctypes.POINTER(c_mlp_frame), vp, vp, vp, vp, ctypes.POINTER(vp)]
    L.lt_destroy_mlp.restype = None
    L.lt_destroy_mlp.argtypes = [vp]
    L.lt_mlp_stats_get.restype = st
    L.lt_mlp_stats_get.argtypes = [vp, ctypes.POINTER(c_mlp_stats)]
    L.lt_mlp_get_params.restype = st
    L.lt_mlp_get_params.argtypes = [vp, vp, vp]
    L.lt_mlp_query.restype = st
    L.lt_mlp_query.argtypes = [vp, ctypes.POINTER(c_rays_in), vp, ctypes.POINTER(c_rays_out),
                               ctypes.c_size_t, ctypes.c_int32, vp]
    L.lt_mlp_grad.restype = st
    L.lt_mlp_grad.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_int32, vp,
                              ctypes.POINTER(ctypes.c_double)]
    L.lt_mlp_features.restype = st
    L.lt_mlp_features.argtypes = [vp, ctypes.POINTER(c_rays_in), vp, vp, ctypes.c_size_t, vp]


_prev_declare = _declare


def _declare(L: ctypes.CDLL) -> None:  # noqa: F811
    _prev_declare(L)
    _declare_mlp(L)
    _declare_paths(L)


def mlp_frame(path_id: int, rho: float, wmax: float, lam_lo: float = 380.0,
              lam_hi: float = 780.0) -> c_mlp_frame:
    return c_mlp_frame(path_id, rho, wmax, lam_lo, lam_hi)


class Mlp:
    """A learned map resident on the device."""

    def __init__(self, handle):
        self.handle = handle

    @classmethod
    def create(cls, lens: Lens, frame: c_mlp_frame, reg, cls_params, t_mean, t_std) -> "Mlp":
        import numpy as np
        reg = np.ascontiguousarray(reg, np.float32)
        cp = np.ascontiguousarray(cls_params, np.float32)
        tm = np.ascontiguousarray(t_mean, np.float64)
        ts = np.ascontiguousarray(t_std, np.float64)
        h = ctypes.c_void_p()
        check(lib().lt_mlp_create(lens.handle, ctypes.byref(frame), reg.ctypes.data, cp.ctypes.data,
                                  tm.ctypes.data, ts.ctypes.data, ctypes.byref(h)))
        return cls(h)

    @classmethod
    def train(cls, lens: Lens, frame: c_mlp_frame, fit, init_reg, init_cls, reg_steps=2000,
              reg_batch=8192, cls_steps=2000, cls_batch=8192, lr=1e-4, lr_decay=0.95,
              decay_every=10000, ft_steps=0, ft_batch=8192, ft_lr=1e-6, seed=1,
              stream=None, n_fit_uniform=None) -> "Mlp":
        """fit: a batch.DeviceRays (or FitRays) of training rays; init_*: host
        FP32 parameters.  n_fit_uniform defaults to the fit set's own
        (FitRays from valid_region_fit carry it; 0 otherwise)."""
        import numpy as np
        ir = np.ascontiguousarray(init_reg, np.float32)
        ic = np.ascontiguousarray(init_cls, np.float32)
        o = c_mlp_opts()
        o.frame = frame
        o.fit_x, o.fit_y, o.fit_dx, o.fit_dy, o.fit_dz = [_ptr(t) for t in fit.inp]
        o.fit_lambda = _ptr(fit.lam)
        o.n_fit = fit.n
        o.init_reg, o.init_cls = ir.ctypes.data, ic.ctypes.data
        o.reg_steps, o.reg_batch, o.cls_steps, o.cls_batch = reg_steps, reg_batch, cls_steps, cls_batch
        o.lr, o.lr_decay, o.decay_every = lr, lr_decay, decay_every
        o.ft_steps, o.ft_batch, o.ft_lr = ft_steps, ft_batch, ft_lr
        o.seed = seed
        o.n_fit_uniform = getattr(fit, "n_uniform", 0) if n_fit_uniform is None else n_fit_uniform
        h = ctypes.c_void_p()
        check(lib().lt_mlp_train(lens.handle, ctypes.byref(o), ctypes.byref(h), _stream_handle(stream)))
        return cls(h)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().lt_destroy_mlp(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = c_mlp_stats()
        check(lib().lt_mlp_stats_get(self.handle, ctypes.byref(s)))
        return {"n_train": s.n_train, "n_valid": s.n_valid, "reg_loss": s.reg_loss,
                "cls_loss": s.cls_loss, "t_mean": list(s.t_mean), "t_std": list(s.t_std),
                "train_ms": s.train_ms, "tc_wait_timeouts": s.tc_wait_timeouts,
                "n_valid_uniform": s.n_valid_uniform, "cls_prior_shift": s.cls_prior_shift}

    def params(self):
        import numpy as np
        reg = np.empty(MLP_REG_PARAMS, np.float32)
        cp = np.empty(MLP_CLS_PARAMS, np.float32)
        check(lib().lt_mlp_get_params(self.handle, reg.ctypes.data, cp.ctypes.data))
        return reg, cp

    def query(self, inp: Sequence, lam, out: Sequence, n: int, precision: int = MLP_F32,
              stream=None) -> None:
        ri = rays_in(*inp)
        ro = rays_out(*out)
        check(lib().lt_mlp_query(self.handle, ctypes.byref(ri), _ptr(lam), ctypes.byref(ro), n,
                                 precision, _stream_handle(stream)))

    def grad(self, net: int, X, targets, B: int):
        """(gradient FP64 numpy array, loss) of one batch; X, targets: device tensors."""
        import numpy as np
        g = np.zeros(MLP_REG_PARAMS if net == 0 else MLP_CLS_PARAMS, np.float64)
        loss = ctypes.c_double()
        check(lib().lt_mlp_grad(self.handle, net, _ptr(X), _ptr(targets), B, g.ctypes.data,
                                ctypes.byref(loss)))
        return g, loss.value

    def features(self, inp: Sequence, lam, X, n: int, stream=None) -> None:
        ri = rays_in(*inp)
        check(lib().lt_mlp_features(self.handle, ctypes.byref(ri), _ptr(lam), _ptr(X), n,
                                    _stream_handle(stream)))


def flat_params(params) -> "np.ndarray":
    """Oracle-style [(W, b), ...] (W: out x in) -> the library's flat FP32 layout."""
    import numpy as np
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def unflat_params(flat, sizes):
    """The library's flat layout -> [(W, b), ...] in FP64 for layer sizes [in, h, ..., out]."""
    import numpy as np
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(flat[o:o + a * b], np.float64).reshape(b, a)
        o += a * b
        bb = np.asarray(flat[o:o + b], np.float64)
        o += b
        out.append((W, bb))
    return out


# ------------------------------------------------------------------ serving

REQ_TRACE, REQ_QUERY, REQ_MLP = 0, 1, 2
REQ_HOST_BUFFERS = 0x1
OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, ENOTREADY = 0, -1, -2, -3, -4, -5, -6


class c_server_opts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("n_streams", ctypes.c_int32),
                ("fuse_max_requests", ctypes.c_int32), ("fuse_max_rays", ctypes.c_size_t),
                ("inject_fail_every", ctypes.c_int32), ("batch_window_us", ctypes.c_uint32)]


class c_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("lens", ctypes.c_void_p), ("path_id", ctypes.c_int32),
                ("map", ctypes.c_void_p), ("query_mode", ctypes.c_int32),
                ("mlp", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("inp", c_rays_in), ("lambda_nm", ctypes.c_void_p), ("out", c_rays_out),
                ("n", ctypes.c_size_t), ("deadline_us", ctypes.c_uint32)]


class c_ticket_info(ctypes.Structure):
    _fields_ = [("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("fused", ctypes.c_int32)]


class c_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "failed", "timed_out",
                                               "launches", "fused_launches", "fused_requests",
                                               "rays")] + \
               [("bytes_in_flight", ctypes.c_size_t), ("peak_bytes_in_flight", ctypes.c_size_t)]


def _declare_server(L: ctypes.CDLL) -> None:
    vp = ctypes.c_void_p
    L.lt_server_create.restype = ctypes.c_int
    L.lt_server_create.argtypes = [ctypes.POINTER(c_server_opts), ctypes.POINTER(vp)]
    L.lt_server_destroy.restype = None
    L.lt_server_destroy.argtypes = [vp]
    L.lt_submit.restype = ctypes.c_int
    L.lt_submit.argtypes = [vp, ctypes.POINTER(c_request), ctypes.POINTER(ctypes.c_uint64)]
    L.lt_poll.restype = ctypes.c_int
    L.lt_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32]
    L.lt_poll_info.restype = ctypes.c_int
    L.lt_poll_info.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(c_ticket_info)]
    L.lt_server_stats_get.restype = ctypes.c_int
    L.lt_server_stats_get.argtypes = [vp, ctypes.POINTER(c_server_stats)]


_prev_declare_srv = _declare


def _declare(L: ctypes.CDLL) -> None:  # noqa: F811
    _prev_declare_srv(L)
    _declare_server(L)


class Server:
    """lt_server: submit trace / query / learned-map requests, poll tickets."""

    def __init__(self, mem_budget_bytes=0, n_streams=0, fuse_max_requests=0, fuse_max_rays=0,
                 inject_fail_every=0, batch_window_us=0):
        o = c_server_opts(mem_budget_bytes, n_streams, fuse_max_requests, fuse_max_rays,
                          inject_fail_every, batch_window_us)
        self.handle = ctypes.c_void_p()
        check(lib().lt_server_create(ctypes.byref(o), ctypes.byref(self.handle)))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().lt_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, kind, inp, lam, out, n, lens=None, path_id=0, gmap=None, query_mode=0,
                mlp=None, precision=0, deadline_us=0, host=False) -> int:
        r = c_request()
        r.kind = kind
        r.flags = REQ_HOST_BUFFERS if host else 0
        r.lens = lens.handle if lens is not None else None
        r.path_id = path_id
        r.map = gmap.handle if gmap is not None else None
        r.query_mode = query_mode
        r.mlp = mlp.handle if mlp is not None else None
        r.precision = precision
        r.inp = rays_in(*inp)
        r.lambda_nm = _ptr(lam)
        r.out = rays_out(*out)
        r.n = n
        r.deadline_us = deadline_us
        t = ctypes.c_uint64()
        check(lib().lt_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def submit_trace(self, lens, inp, lam, path_id, out, n, **kw) -> int:
        return self._submit(REQ_TRACE, inp, lam, out, n, lens=lens, path_id=path_id, **kw)

    def submit_query(self, gmap, inp, lam, out, n, query_mode=QUERY_TABLE, **kw) -> int:
        return self._submit(REQ_QUERY, inp, lam, out, n, gmap=gmap, query_mode=query_mode, **kw)

    def submit_mlp(self, mlp, inp, lam, out, n, precision=MLP_F32, **kw) -> int:
        return self._submit(REQ_MLP, inp, lam, out, n, mlp=mlp, precision=precision, **kw)

    def poll(self, ticket: int, timeout_us: int = 0):
        """(status, info dict or None): status is the raw lt_status."""
        info = c_ticket_info()
        st = lib().lt_poll_info(self.handle, ticket, timeout_us, ctypes.byref(info))
        if st in (ENOTREADY, EINVAL):
            return st, None
        return st, {"queue_us": info.queue_us, "latency_us": info.latency_us, "fused": info.fused}

    def wait(self, ticket: int, timeout_us: int = 60_000_000) -> dict:
        st, info = self.poll(ticket, timeout_us)
        check(st)
        return info

    def stats(self) -> dict:
        s = c_server_stats()
        check(lib().lt_server_stats_get(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in c_server_stats._fields_}
