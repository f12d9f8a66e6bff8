"""lt_trace_paths (the flare workload of Sec. 4.2: main path plus every
two-bounce ghost of the 11-surface lens, one launch, wavelength redrawn per
path) against the oracle, element by element after undoing the compaction.

The order of entries inside a path's segment is not unique (warps append in
whatever order they finish); what is unique -- the set of ray indices that
reached the image and each one's outputs -- is compared, and the entries are
checked to be distinct, in range and within the counter."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import compare_trace

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


def flare_lambdas(n_paths, n):
    return np.stack([w.flare_wavelengths(p, n) for p in range(n_paths)])


def uncompact(po, p, n):
    """Scatter path p's entries back to [n] arrays (zeros, flag 0 where absent)."""
    idx, out, flags = po.path(p)
    assert len(np.unique(idx)) == len(idx), "a ray was written twice"
    assert (idx < n).all()
    full = np.zeros((n, 6), np.float32)
    fl = np.zeros(n, np.uint8)
    full[idx] = out
    fl[idx] = flags
    assert (flags & lt.FLAG_VALID).all()
    return full, fl


def run_paths(lens, rays, lam2d, path_ids, capacity, lam_stride=None):
    n = len(rays)
    d = batch.DeviceRays(rays)
    lam = torch.from_numpy(np.ascontiguousarray(lam2d, np.float32).reshape(-1)).cuda()
    po = batch.PathsOut(len(path_ids), capacity)
    lt.trace_paths(lens, d.inp, lam, n if lam_stride is None else lam_stride, path_ids, po, n)
    torch.cuda.synchronize()
    return po


def test_every_flare_path_matches_oracle(eleven):
    lens = lt.Lens(eleven)
    ol = oracle.Lens(eleven)
    n = 3000                                  # 11 full tiles and a ragged one
    rays = w.flare_rays(eleven, n)
    P = lens.n_paths
    lam = flare_lambdas(P, n)
    po = run_paths(lens, rays, lam, list(range(P)), n)
    counts = po.counts()
    total_or = 0
    for p in range(P):
        full, fl = uncompact(po, p, n)
        rp = dataclasses.replace(rays, lam=lam[p])
        path = oracle.path_ij(eleven.n_surfaces, p)
        ex, ev, edge, kmin = ol.trace(rp, path)
        assert counts[p] == int(((fl & lt.FLAG_VALID) != 0).sum())
        compare_trace(full, fl, ex, ev, edge, kmin, f"paths {p}", cond=(ol, rp, path))
        total_or += int((ev == 1).sum())
    print("valid per path", counts.tolist(), "total", counts.sum(), "oracle", total_or)
    assert counts[0] > 0.1 * n


def test_identical_to_single_path_trace(eleven):
    """Shared wavelengths (stride 0), repeated paths: every entry equals
    lt_trace of the same ray bit for bit, flags included."""
    lens = lt.Lens(eleven)
    n = 5000
    rays = w.flare_rays(eleven, n)
    ids = [0, 5, 17, 0, 54]
    po = run_paths(lens, rays, rays.lam[None, :], ids, n, lam_stride=0)
    d = batch.DeviceRays(rays)
    for k, pid in enumerate(ids):
        o = batch.DeviceOut(n)
        lt.trace(lens, d.inp, d.lam, pid, o.out, n)
        torch.cuda.synchronize()
        ref, rf = o.numpy()
        full, fl = uncompact(po, k, n)
        v = (rf & lt.FLAG_VALID) != 0
        assert np.array_equal(fl[v], rf[v]) and not fl[~v].any()
        assert np.array_equal(full.view(np.uint32), ref.view(np.uint32)), pid


def test_capacity_overflow_counts_everything(eleven):
    lens = lt.Lens(eleven)
    n = 4096
    rays = w.flare_rays(eleven, n)
    po = run_paths(lens, rays, rays.lam[None, :], [0], 100, lam_stride=0)
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(n)
    lt.trace(lens, d.inp, d.lam, 0, o.out, n)
    torch.cuda.synchronize()
    ref, rf = o.numpy()
    assert po.counts()[0] == int(((rf & lt.FLAG_VALID) != 0).sum()) > 100
    idx, out, flags = po.path(0)
    assert len(idx) == 100 and len(np.unique(idx)) == 100
    assert np.array_equal(out.view(np.uint32), ref[idx].view(np.uint32))


def test_zero_rays_zeroes_counters(eleven):
    lens = lt.Lens(eleven)
    po = batch.PathsOut(3, 4)
    po.valid_count.fill_(7)
    d = batch.DeviceRays(w.flare_rays(eleven, 4))
    lt.trace_paths(lens, d.inp, d.lam, 0, [0, 1, 2], po, 0)
    torch.cuda.synchronize()
    assert (po.counts() == 0).all()


def test_bad_arguments(eleven):
    lens = lt.Lens(eleven)
    d = batch.DeviceRays(w.flare_rays(eleven, 64))
    po = batch.PathsOut(2, 64)
    with pytest.raises(lt.LTError):
        lt.trace_paths(lens, d.inp, d.lam, 0, [0, lens.n_paths], po, 64)
    with pytest.raises(lt.LTError):
        lt.trace_paths(lens, d.inp, d.lam, 0, [], po, 64)
    po.capacity = 0
    with pytest.raises(lt.LTError):
        lt.trace_paths(lens, d.inp, d.lam, 0, [0, 1], po, 64)


def test_full_size_flare_launch_sampled(eleven):
    """The full flare workload (56 paths x 1,048,576 rays, one launch, as the
    benchmark runs it), checked on 400 sampled rays per path."""
    lens = lt.Lens(eleven)
    ol = oracle.Lens(eleven)
    rays = w.flare_rays(eleven)
    n = len(rays)
    P = lens.n_paths
    lam = flare_lambdas(P, n)
    po = run_paths(lens, rays, lam, list(range(P)), n)
    counts = po.counts()
    rng = np.random.Generator(np.random.PCG64(99))
    for p in range(P):
        lo = p * n
        k = int(counts[p])
        idx = po.ray_index[lo:lo + k].long()
        inv = torch.full((n,), -1, dtype=torch.long, device="cuda")
        inv[idx] = torch.arange(k, device="cuda")
        s = np.sort(rng.choice(n, 400, replace=False))
        pos = inv[torch.from_numpy(s).cuda()].cpu().numpy()
        out = np.zeros((len(s), 6), np.float32)
        fl = np.zeros(len(s), np.uint8)
        hit = pos >= 0
        if hit.any():
            g = torch.from_numpy(pos[hit] + lo).cuda()
            out[hit] = torch.stack([t[g] for t in po.f], dim=1).cpu().numpy()
            fl[hit] = po.flags[g].cpu().numpy()
        rp = dataclasses.replace(rays.subset(s), lam=lam[p][s])
        path = oracle.path_ij(eleven.n_surfaces, p)
        ex, ev, edge, kmin = ol.trace(rp, path)
        compare_trace(out, fl, ex, ev, edge, kmin, f"full paths {p}", cond=(ol, rp, path))
    print("full-size valid counts", counts.tolist(), "total", int(counts.sum()))
