"""The allocation-free map query (lt_query_noalloc).

Some callers of this library cannot allocate GPU memory while they run: a
renderer or serving process whose allocator reserves the whole device at
start-up, or a loop where cudaMalloc (and the synchronisation it can imply)
is not allowed.  lt_query_noalloc gives them the map query with its trace
queue in a fixed array inside the library instead of the memory pool.  This
checks, through the C ABI, that it answers like lt_query on two calls in a
row (the array keeps the first call's contents, so the second call shows
that the counter is cleared), that the device's free memory is the same
before and after its calls (nothing was allocated), and that it refuses
batches larger than the array.  The file is named to run last: if it fails,
every other test has run.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_04017_gb300 import batch, lt, workloads as w

from parity import DIR_TOL, I_TOL, POS_TOL

pytestmark = pytest.mark.gpu


def test_noalloc_query_matches_lt_query_on_two_calls():
    p = w.singlet_lens()
    sm = math.tan(math.radians(10.0))
    lo, hi = [-12, -12, -sm, -sm, 380.0], [12, 12, sm, sm, 780.0]
    fit = w.singlet_rays()
    gmap = lt.Map.build(lt.Lens(p), 0, [16, 16, 16, 16, 4], lo, hi, fit=batch.DeviceRays(fit))
    for call, (n, seed) in enumerate([(300001, 11), (65537, 12)]):
        rays = w.entrance_rays(n, seed, 12.5)       # a few rays fall outside the box
        d = batch.DeviceRays(rays)
        ref = batch.DeviceOut(n)
        gmap.query(d.inp, d.lam, ref.out, n)
        got = batch.DeviceOut(n)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        lt.query_noalloc(gmap, d.inp, d.lam, got.out, n)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, f"call {call}: device memory was allocated"
        ro, rf = ref.numpy()
        go, gf = got.numpy()
        assert np.array_equal(gf, rf), f"call {call}: flags differ"
        assert np.abs(go[:, 0:2] - ro[:, 0:2]).max() <= POS_TOL
        assert np.abs(go[:, 2:5] - ro[:, 2:5]).max() <= DIR_TOL
        assert np.abs(go[:, 5] - ro[:, 5]).max() <= I_TOL
        assert ((gf & lt.FLAG_TRACED) != 0).sum() > 1000


def test_noalloc_rejects_batches_above_its_array():
    p = w.singlet_lens()
    sm = math.tan(math.radians(10.0))
    gmap = lt.Map.build(lt.Lens(p), 0, [3, 3, 3, 3, 2], [-12, -12, -sm, -sm, 380.0],
                        [12, 12, sm, sm, 780.0])
    n = lt.NOALLOC_MAX_RAYS + 1
    d = batch.DeviceRays(w.singlet_rays(n))
    o = batch.DeviceOut(n)
    with pytest.raises(lt.LTError) as e:
        lt.query_noalloc(gmap, d.inp, d.lam, o.out, n)
    assert e.value.code == lt.LT_EINVAL and "LT_NOALLOC_MAX_RAYS" in str(e.value)
