"""lt_splat_paths (forward light tracing onto the sensor, Sec. 3, Eq. 8)
against the oracle's FP64 trace and splat, pixel by pixel.

A pixel of the GPU image is a sum of FP32 atomic adds in no fixed order,
and each deposit rests on an FP32 trace within the tracer's tolerances.
The per-pixel bound is therefore the oracle's deposit_bound for those
tolerances (position 1e-4 mm, I and d_z 1e-6) plus the FP32 accumulation
of the pixel's deposits.  Rays the tolerances do not cover (within 1e-6 mm
of an aperture edge, or refracting near grazing, k < 1e-2) are left out of
the batch given to both sides.  The image totals are compared as well, which
a wrong factor (a missing G = d_z, say) cannot pass."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import splat as S
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import DIR_TOL, EDGE_EPS, GRAZING_K, I_TOL, POS_TOL

pytestmark = pytest.mark.gpu


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def eleven():
    return w.eleven_surface_lens(oracle_accept)


def gpu_splat(lens, rays, lam2d, path_ids, W, H, px, weight, per_path):
    n = len(rays)
    d = batch.DeviceRays(rays)
    lam = torch.from_numpy(np.ascontiguousarray(lam2d, np.float32).reshape(-1)).cuda()
    img = torch.zeros((len(path_ids) if per_path else 1, H, W), dtype=torch.float32, device="cuda")
    lt.splat_paths(lens, d.inp, lam, n, path_ids, n, W, H, px, img, weight=weight, per_path=per_path)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64)


def well_conditioned(ol, rays, path):
    _, valid, edge, kmin = ol.trace(rays, path)
    return ~((edge < EDGE_EPS) | (kmin < GRAZING_K))


def check_image(gpu, ol, rays, path, W, H, px, weight, label):
    out, valid, _, _ = ol.trace(rays, path)
    v = valid == 1
    ref = S.splat(out[:, 0], out[:, 1], out[:, 4], out[:, 5], v, W, H, px, weight)
    bound = S.deposit_bound(out[:, 0], out[:, 1], out[:, 4], out[:, 5], v, W, H, px, weight,
                            POS_TOL, max(DIR_TOL, I_TOL))
    # FP32 accumulation of the pixel's deposits (a few ulps of the running sum each)
    mag = S.splat(out[:, 0], out[:, 1], np.abs(out[:, 4]), np.abs(out[:, 5]), v, W, H, px, abs(weight))
    tol = bound + 4e-7 * mag * np.maximum(1.0, np.sqrt(max(1, v.sum()) / (W * H))) + 1e-12
    err = np.abs(gpu - ref)
    assert (err <= tol).all(), f"{label}: pixel error {err.max()} over bound {tol[err.argmax() // W, err.argmax() % W]}"
    assert ref.sum() > 0.0, f"{label}: nothing reached the sensor"
    assert abs(gpu.sum() - ref.sum()) <= bound.sum() + 1e-6 * mag.sum(), f"{label}: totals differ"
    return err.max(), ref.sum()


@pytest.mark.parametrize("path_id", [0, 1])
def test_singlet_paths_match_oracle(path_id):
    p = w.singlet_lens()
    lens, ol = lt.Lens(p), oracle.Lens(p)
    path = oracle.path_ij(2, path_id)
    rays = w.singlet_rays(20000)
    rays = rays.subset(np.nonzero(well_conditioned(ol, rays, path))[0])
    W, H, px = 96, 64, 0.25                     # a 24 x 16 mm sensor
    weight = 1.0 / len(rays)
    gpu = gpu_splat(lens, rays, rays.lam[None, :], [path_id], W, H, px, weight, False)[0]
    e, tot = check_image(gpu, ol, rays, path, W, H, px, weight, f"singlet path {path_id}")
    print("singlet splat", path_id, "max pixel error", e, "total", tot)


def test_eleven_surface_flare_paths_match_oracle(eleven):
    lens, ol = lt.Lens(eleven), oracle.Lens(eleven)
    S_ = eleven.n_surfaces
    pids = [0, 1, 7, 20, 33, 54, 55]
    base = w.eleven_rays(eleven, 12000)
    W, H, px = 120, 80, 0.2
    for pid in pids:
        path = oracle.path_ij(S_, pid)
        lam = w.flare_wavelengths(pid, len(base))
        rays = w.Rays(base.x, base.y, base.dx, base.dy, base.dz, lam.astype(np.float32))
        rays = rays.subset(np.nonzero(well_conditioned(ol, rays, path))[0])
        weight = 1.0 / len(rays)
        gpu = gpu_splat(lens, rays, rays.lam[None, :], [pid], W, H, px, weight, False)[0]
        e, tot = check_image(gpu, ol, rays, path, W, H, px, weight, f"eleven path {pid}")
        print("eleven splat", pid, "max pixel error", e, "total", tot)


def test_one_launch_over_many_paths_equals_per_path_images(eleven):
    """All 56 paths in one call: per-path images (per_path = 1) agree with one
    call per path, and the summed image (per_path = 0) with their sum, within
    the FP32 reordering of the atomic adds."""
    lens = lt.Lens(eleven)
    n = 4096
    rays = w.eleven_rays(eleven, n)
    pids = list(range(lens.n_paths))
    lam2d = np.stack([w.flare_wavelengths(p, n) for p in pids]).astype(np.float32)
    W, H, px = 64, 64, 0.4
    per = gpu_splat(lens, rays, lam2d, pids, W, H, px, 1.0, True)
    summed = gpu_splat(lens, rays, lam2d, pids, W, H, px, 1.0, False)[0]
    for k in (0, 1, 30, 55):
        one = gpu_splat(lens, rays, lam2d[k][None, :], [pids[k]], W, H, px, 1.0, False)[0]
        np.testing.assert_allclose(per[k], one, rtol=1e-5, atol=1e-6 * max(1.0, one.max()))
    np.testing.assert_allclose(summed, per.sum(axis=0), rtol=1e-5, atol=1e-6 * max(1.0, summed.max()))
    assert per[0].sum() > per[1:].sum(axis=(1, 2)).max()    # the main path carries the most light


def test_accumulates_into_the_image():
    p = w.singlet_lens()
    lens = lt.Lens(p)
    rays = w.singlet_rays(5000)
    W, H, px = 16, 16, 0.1                      # a 1.6 mm sensor: most rays miss it
    a = gpu_splat(lens, rays, rays.lam[None, :], [0], W, H, px, 1.0, False)[0]
    d = batch.DeviceRays(rays)
    img = torch.from_numpy(np.stack([a]).astype(np.float32)).cuda()
    lt.splat_paths(lens, d.inp, d.lam, len(rays), [0], len(rays), W, H, px, img)
    torch.cuda.synchronize()
    np.testing.assert_allclose(img.cpu().numpy()[0], 2 * a, rtol=1e-5, atol=1e-6)
    assert a.sum() > 0.0
