"""CPU checks of the C ABI: the library loads, exports every function the
headers declare, validates arguments before touching the GPU, and its host
logic (paraxial image plane, path numbering) agrees with the oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_2605_04017_gb300 import lt, workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(lt_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function():
    L = lt.lib()
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_built_for_sm103a_only():
    from paper_2605_04017_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_paraxial_matches_oracle(which):
    p = w.singlet_lens() if which == "singlet" else w.eleven_surface_lens(oracle_accept)
    L = lt.Lens(p)
    O = oracle.Lens(p)
    for lam in (380.0, 587.6, 780.0):
        efl, bfd, zi = L.paraxial(lam)
        oe, ob = O.paraxial(lam)
        assert efl == pytest.approx(oe, rel=1e-12)
        assert bfd == pytest.approx(ob, rel=1e-12)
    assert zi == pytest.approx(O.z_image(), rel=1e-13)


def test_path_numbering_matches_oracle():
    for S in (2, 5, 11, 22):
        L_paths = 1 + S * (S - 1) // 2
        for pid in range(L_paths):
            ij = lt.path_ij(S, pid)
            assert ij == oracle.path_ij(S, pid)
            assert lt.path_id(S, *ij) == pid
            assert lt.path_code(S, *ij) == oracle.path_code(S, *ij)
    assert lt.path_code(13, 1, 3) == 131092
    assert lt.path_code(12, 3, 5) == 65616
    assert lt.path_id(5, 3, 2) == -1


def test_lens_validation():
    p = w.singlet_lens()
    p.surfaces[0].aperture_r = 60.0        # larger than |R| = 50
    with pytest.raises(lt.LTError) as e:
        lt.Lens(p)
    assert e.value.code == lt.LT_EBADLENS
    p = w.singlet_lens()
    p.surfaces[0].glass_after = 3
    with pytest.raises(lt.LTError) as e:
        lt.Lens(p)
    assert e.value.code == lt.LT_EBADLENS
    # a diverging lens has no real paraxial focus behind it
    p = w.singlet_lens()
    p.surfaces[0].curvature = -1 / 50.0
    p.surfaces[1].curvature = 1 / 50.0
    with pytest.raises(lt.LTError):
        lt.Lens(p)
    assert "back focal" in lt.last_error()
    p = w.singlet_lens()
    p.surfaces = p.surfaces * 20           # 40 surfaces > LT_MAX_SURFACES
    with pytest.raises(lt.LTError) as e:
        lt.Lens(p)
    assert e.value.code == lt.LT_EINVAL


def test_trace_argument_errors_without_gpu():
    L = lt.Lens(w.singlet_lens())
    ri = lt.c_rays_in()
    ro = lt.c_rays_out()
    # NULL arrays with n > 0
    rc = lt.lib().lt_trace(L.handle, ctypes.byref(ri), None, 0, ctypes.byref(ro), 10, None)
    assert rc == lt.LT_EINVAL
    # bad path id
    rc = lt.lib().lt_trace(L.handle, ctypes.byref(ri), None, 2, ctypes.byref(ro), 0, None)
    assert rc == lt.LT_EINVAL and "path" in lt.last_error()
    # misaligned arrays
    buf = np.zeros(64, np.float32)
    base = buf.ctypes.data
    ri = lt.c_rays_in(base + 4, base, base, base, base)
    ro = lt.c_rays_out(base, base, base, base, base, base, base)
    rc = lt.lib().lt_trace(L.handle, ctypes.byref(ri), base, 0, ctypes.byref(ro), 4, None)
    assert rc == lt.LT_EINVAL and "aligned" in lt.last_error()
    # n = 0 is a no-op
    rc = lt.lib().lt_trace(L.handle, ctypes.byref(lt.c_rays_in()), None, 0,
                           ctypes.byref(lt.c_rays_out()), 0, None)
    assert rc == lt.LT_OK


def test_trace_paths_argument_errors_without_gpu():
    L = lt.Lens(w.singlet_lens())
    ri = lt.c_rays_in()
    po = lt.c_paths_out()
    ids = (ctypes.c_int32 * 2)(0, 1)
    f = lt.lib().lt_trace_paths
    assert f(None, ctypes.byref(ri), None, 0, ids, 2, ctypes.byref(po), 0, None) == lt.LT_EINVAL
    po.capacity = 4
    po.valid_count = 16
    assert f(L.handle, ctypes.byref(ri), None, 0, ids, 0, ctypes.byref(po), 0, None) == lt.LT_EINVAL
    bad = (ctypes.c_int32 * 1)(2)          # the singlet has paths 0 and 1 only
    assert f(L.handle, ctypes.byref(ri), None, 0, bad, 1, ctypes.byref(po), 0, None) == lt.LT_EINVAL
    assert "path" in lt.last_error()
    po.capacity = 0
    assert f(L.handle, ctypes.byref(ri), None, 0, ids, 2, ctypes.byref(po), 0, None) == lt.LT_EINVAL


def test_splat_paths_argument_errors_without_gpu():
    L = lt.Lens(w.singlet_lens())
    ri = lt.c_rays_in()
    ids = (ctypes.c_int32 * 2)(0, 1)
    sen = lt.c_sensor(64, 48, 0.05, 1.0, 0)
    f = lt.lib().lt_splat_paths
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(lt.c_rays_in), ctypes.c_void_p, ctypes.c_size_t,
                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(lt.c_sensor),
                  ctypes.c_void_p, ctypes.c_void_p]
    img = 256
    assert f(L.handle, ctypes.byref(ri), None, 0, ids, 2, 0, None, img, None) == lt.LT_EINVAL
    bad = lt.c_sensor(0, 48, 0.05, 1.0, 0)
    assert f(L.handle, ctypes.byref(ri), None, 0, ids, 2, 0, ctypes.byref(bad), img, None) == lt.LT_EINVAL
    assert "sensor" in lt.last_error()
    bad = lt.c_sensor(64, 48, 0.0, 1.0, 0)
    assert f(L.handle, ctypes.byref(ri), None, 0, ids, 2, 0, ctypes.byref(bad), img, None) == lt.LT_EINVAL
    nopath = (ctypes.c_int32 * 1)(2)          # the singlet has paths 0 and 1 only
    assert f(L.handle, ctypes.byref(ri), None, 0, nopath, 1, 0, ctypes.byref(sen), img, None) == lt.LT_EINVAL
    # n = 0 deposits nothing and succeeds without touching the device
    assert f(L.handle, ctypes.byref(ri), None, 0, ids, 2, 0, ctypes.byref(sen), img, None) == lt.LT_OK


@pytest.mark.parametrize("which", ["singlet", "eleven"])
def test_reversed_lens_matches_oracle_reversal(which):
    """lt_reverse_lens (host code) against the oracle's own reversal: focal
    length and image plane, for the in-focus and a refocused sensor."""
    from oracle import reverse as R
    p = w.singlet_lens() if which == "singlet" else w.eleven_surface_lens(oracle_accept)
    L = lt.Lens(p)
    zi = L.paraxial(587.6)[2]
    for sensor_z, out_z in ((zi, 0.0), (zi + 0.6, -2.0)):
        back = L.reversed(sensor_z, out_z)
        ob = oracle.Lens(R.reverse_prescription(p, sensor_z, out_z, w.IMAGE_ABS))
        for lam in (400.0, 587.6, 760.0):
            e, b, z = back.paraxial(lam)
            oe, obf = ob.paraxial(lam)
            assert e == pytest.approx(oe, rel=1e-12) and b == pytest.approx(obf, rel=1e-12)
        assert z == pytest.approx(ob.z_image(), abs=1e-12)
        assert back.paraxial(587.6)[0] == pytest.approx(L.paraxial(587.6)[0], rel=1e-12)


def test_reverse_lens_argument_errors():
    L = lt.Lens(w.singlet_lens())
    zi = L.paraxial(587.6)[2]
    f = lt.lib().lt_reverse_lens
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert f(None, zi, 0.0, ctypes.byref(h)) == lt.LT_EINVAL
    assert f(L.handle, 4.0, 0.0, ctypes.byref(h)) == lt.LT_EINVAL        # sensor inside the lens
    assert "sensor" in lt.last_error()
    assert f(L.handle, zi, 1.0, ctypes.byref(h)) == lt.LT_EINVAL         # output plane behind surface 1
    assert f(L.handle, zi, float("nan"), ctypes.byref(h)) == lt.LT_EINVAL
    assert not h.value


def test_server_entry_points_without_gpu():
    import torch
    t = ctypes.c_uint64()
    assert lt.lib().lt_submit(None, None, ctypes.byref(t)) == lt.LT_EINVAL
    assert lt.lib().lt_poll(None, 1, 0) == lt.LT_EINVAL
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    rc = lt.lib().lt_server_create(None, ctypes.byref(h))
    assert rc != lt.LT_OK and not h.value


def test_map_load_rejects_files_that_are_not_maps(tmp_path):
    # missing, empty, wrong magic and truncated files are refused with
    # LT_EIO before any device memory is touched
    missing = tmp_path / "none.ltmap"
    empty = tmp_path / "empty.ltmap"
    empty.write_bytes(b"")
    wrong = tmp_path / "wrong.ltmap"
    wrong.write_bytes(b"NOTAMAP\0" + bytes(4096))
    trunc = tmp_path / "trunc.ltmap"
    trunc.write_bytes(b"LTMAP01\0" + (2).to_bytes(4, "little") + bytes(16))
    for f in (missing, empty, wrong, trunc):
        with pytest.raises(lt.LTError) as e:
            lt.Map.load(str(f))
        assert e.value.code == lt.LT_EIO, f


def test_poly_map_options_rejected_before_the_gpu():
    """lt_build_poly_map validates its options on the host (no device needed)."""
    import math
    lens = lt.Lens(w.singlet_lens())
    smax = math.tan(math.radians(10)) * math.sqrt(2)
    good = dict(path_id=0, rho=12.0, smax=smax, degree=3, patches=(2, 2, 1, 1), cells=(2, 2, 2, 1), samples=5)
    bad = [dict(degree=0), dict(degree=lt.POLY_MAX_DEGREE + 1), dict(samples=3), dict(samples=9),
           dict(patches=(0, 1, 1, 1)), dict(cells=(1, 1, 1, 0)), dict(patches=(64, 1, 1, 1), cells=(65, 1, 1, 1)),
           dict(rho=0.0), dict(smax=-1.0), dict(path_id=7), dict(lam=(780.0, 380.0))]
    for b in bad:
        a = dict(good, **b)
        lam = a.pop("lam", (380.0, 780.0))
        with pytest.raises(lt.LTError) as e:
            lt.Map.build_poly(lens, a["path_id"], a["rho"], a["smax"], a["degree"], a["patches"],
                              a["cells"], a["samples"], lam_lo=lam[0], lam_hi=lam[1], stream=0)
        assert e.value.code == -1, (b, e.value)
    # a table map has no polynomial fit to report
    h = ctypes.c_void_p()
    assert lt.lib().lt_poly_stats_get(h, None) == -1


def test_binding_constants_match_the_header():
    src = open(os.path.join(ROOT, "include", "lt.h")).read()
    m = re.search(r"#define LT_NOALLOC_MAX_RAYS \(1 << (\d+)\)", src)
    assert m and lt.NOALLOC_MAX_RAYS == 1 << int(m.group(1))
    m = re.search(r"#define LT_POLY_MAX_DEGREE (\d+)", src)
    assert m and lt.POLY_MAX_DEGREE == int(m.group(1))


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror of a header struct has the C struct's size, and
    each field the two share by name sits at the same offset: the header is
    compiled with the host C compiler and asked for sizeof and offsetof."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    pairs = {}
    for name in dir(lt):
        cls = getattr(lt, name)
        if name.startswith("c_") and isinstance(cls, type) and issubclass(cls, ctypes.Structure):
            cname = "lt_" + name[2:]
            pairs[cname] = cls
    header = open(os.path.join(ROOT, "include", "lt.h")).read()
    pairs = {k: v for k, v in pairs.items() if re.search(r"\}\s*" + k + r"\s*;", header)}
    assert len(pairs) >= 15
    renamed = {"inp": "in"}          # the binding's names for C fields that are Python keywords
    lines = ['#include "lt.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {renamed.get(fname, fname)}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    checked = 0
    for ln in out:
        parts = ln.split()
        if len(parts) != 3:
            continue
        cname, what, val = parts[0], parts[1], int(parts[2])
        cls = pairs[cname]
        if what == "size":
            assert ctypes.sizeof(cls) == val, (cname, ctypes.sizeof(cls), val)
        else:
            assert getattr(cls, what).offset == val, (cname, what, getattr(cls, what).offset, val)
        checked += 1
    assert checked == len(pairs) + sum(len(c._fields_) for c in pairs.values())
