"""The request server (lt_server_create / lt_submit / lt_poll): results of
requests served in a mix (fused trace launches, map queries, learned-map
queries, host-buffer staging, several streams and submitting threads) are
identical, bit for bit, to the same request made alone through lt_trace /
lt_query / lt_mlp_query; memory admission, deadlines, poll waits and launch
failures are exercised on the host (failures are injected by the server's
host-side hook, never by faulting the GPU)."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp as omlp
from paper_2605_04017_gb300 import batch, lt, workloads as w

pytestmark = pytest.mark.gpu


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


@pytest.fixture(scope="module")
def lenses():
    pres = [w.singlet_lens(), w.eleven_surface_lens(oracle_accept)] + \
        w.serving_lenses(oracle_accept, 2)
    return pres, [lt.Lens(p) for p in pres]


@pytest.fixture(scope="module")
def singlet_map(lenses):
    import math
    lens = lenses[1][0]
    sm = math.tan(math.radians(10.0))
    fit = batch.DeviceRays(w.entrance_rays(1 << 18, 5, 12.0))
    return lt.Map.build(lens, 0, [16, 16, 16, 16, 4], [-12, -12, -sm, -sm, 380], [12, 12, sm, sm, 780],
                        fit=fit)


@pytest.fixture(scope="module")
def singlet_mlp(lenses):
    r = np.random.Generator(np.random.PCG64(3))
    reg, cls = omlp.init_params("reg", r), omlp.init_params("cls", r)
    return lt.Mlp.create(lenses[1][0], lt.mlp_frame(0, 12.0, 0.2421), lt.flat_params(reg),
                         lt.flat_params(cls), np.zeros(6), np.ones(6))


def rays_for(pres, n, seed):
    rho = 12.0 if pres.n_surfaces == 2 else w.eleven_rho(pres)
    return w.entrance_rays(n, seed, rho)


def alone(kind, obj, d, n, arg):
    o = batch.DeviceOut(n)
    if kind == lt.REQ_TRACE:
        lt.trace(obj, d.inp, d.lam, arg, o.out, n)
    elif kind == lt.REQ_QUERY:
        obj.query(d.inp, d.lam, o.out, n, arg)
    else:
        obj.query(d.inp, d.lam, o.out, n, arg)
    torch.cuda.synchronize()
    return o.numpy()


def same(a, b):
    (oa, fa), (ob, fb) = a, b
    return np.array_equal(oa.view(np.uint32), ob.view(np.uint32)) and np.array_equal(fa, fb)


def test_mix_matches_alone(lenses, singlet_map, singlet_mlp):
    pres, ls = lenses
    srv = lt.Server(n_streams=3)
    rng = np.random.Generator(np.random.PCG64(17))
    reqs = []
    for k in range(60):
        n = int(rng.choice([1, 37, 256, 1000, 4099, 30000, 65536, 65537, 300000]))
        u = rng.uniform()
        if u < 0.6:
            li = int(rng.integers(len(ls)))
            pid = int(rng.integers(ls[li].n_paths))
            kind, obj, arg, pr = lt.REQ_TRACE, ls[li], pid, pres[li]
        elif u < 0.8:
            kind, obj, arg, pr = lt.REQ_QUERY, singlet_map, lt.QUERY_TABLE, pres[0]
        else:
            kind, obj, arg, pr = lt.REQ_MLP, singlet_mlp, int(rng.integers(4)), pres[0]
        d = batch.DeviceRays(rays_for(pr, n, 1000 + k))
        o = batch.DeviceOut(n)
        reqs.append((kind, obj, arg, d, o, n))
    torch.cuda.synchronize()
    tickets = []
    for kind, obj, arg, d, o, n in reqs:
        if kind == lt.REQ_TRACE:
            t = srv.submit_trace(obj, d.inp, d.lam, arg, o.out, n)
        elif kind == lt.REQ_QUERY:
            t = srv.submit_query(obj, d.inp, d.lam, o.out, n, query_mode=arg)
        else:
            t = srv.submit_mlp(obj, d.inp, d.lam, o.out, n, precision=arg)
        tickets.append(t)
    fused = 0
    for t in tickets:
        info = srv.wait(t)
        fused = max(fused, info["fused"])
    st = srv.stats()
    print("server stats", st, "largest fused launch", fused)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["fused_launches"] >= 1 and fused > 1
    for kind, obj, arg, d, o, n in reqs:
        assert same(o.numpy(), alone(kind, obj, d, n, arg)), (kind, n, arg)
    srv.close()


@pytest.fixture(scope="module")
def eleven_poly_map(lenses):
    import math
    pres, ls = lenses
    rho = w.eleven_rho(pres[1])
    smax = math.tan(math.radians(10.0)) * math.sqrt(2.0)
    return lt.Map.build_poly(ls[1], 0, rho, smax, 3, [4, 4, 2, 1], [8, 8, 8, 4], 5,
                             fit=batch.DeviceRays(w.entrance_rays(1 << 18, 11, rho)), max_residual_mm=1e-4)


def test_fused_every_kind(lenses, singlet_map, singlet_mlp, eleven_poly_map):
    """With a batching window the server holds waiting requests until 96 are
    in: the small traces, table-map queries (both query modes),
    polynomial-patch map queries and learned-map queries of every precision
    each share launches, and every result equals the request made alone, bit
    for bit (ragged sizes, several blocks per request, a tail block)."""
    pres, ls = lenses
    srv = lt.Server(n_streams=2, fuse_max_requests=96, batch_window_us=2_000_000)
    rng = np.random.Generator(np.random.PCG64(23))
    kinds = [(lt.REQ_TRACE, ls[1], 0, pres[1]), (lt.REQ_TRACE, ls[2], 3, pres[2]),
             (lt.REQ_QUERY, singlet_map, lt.QUERY_TABLE, pres[0]),
             (lt.REQ_QUERY, singlet_map, lt.QUERY_NO_MASK, pres[0]),
             (lt.REQ_QUERY, eleven_poly_map, lt.QUERY_TABLE, pres[1])] + \
        [(lt.REQ_MLP, singlet_mlp, p, pres[0]) for p in range(4)]
    reqs = []
    for k in range(96):
        kind, obj, arg, pr = kinds[k % len(kinds)]
        n = int(rng.choice([1, 77, 256, 1023, 1025, 4099, 20000]))
        d = batch.DeviceRays(rays_for(pr, n, 2000 + k))
        reqs.append((kind, obj, arg, d, batch.DeviceOut(n), n))
    torch.cuda.synchronize()
    tickets = []
    for kind, obj, arg, d, o, n in reqs:
        if kind == lt.REQ_TRACE:
            tickets.append(srv.submit_trace(obj, d.inp, d.lam, arg, o.out, n))
        elif kind == lt.REQ_QUERY:
            tickets.append(srv.submit_query(obj, d.inp, d.lam, o.out, n, query_mode=arg))
        else:
            tickets.append(srv.submit_mlp(obj, d.inp, d.lam, o.out, n, precision=arg))
    fused = [srv.wait(t)["fused"] for t in tickets]
    st = srv.stats()
    print("server stats", st)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    # every kind ran fused: the 96 requests fill one window, so each of the 8
    # fusion groups (the two lenses' traces share one) is one launch of all
    # its requests
    for (kind, obj, arg, _), f in zip(kinds, fused[:len(kinds)]):
        assert f > 1, (kind, arg, f)
    assert st["fused_launches"] == 8 and st["fused_requests"] == 96
    for kind, obj, arg, d, o, n in reqs:
        assert same(o.numpy(), alone(kind, obj, d, n, arg)), (kind, n, arg)
    srv.close()


def test_host_buffers(lenses):
    pres, ls = lenses
    srv = lt.Server()
    rays = rays_for(pres[1], 100003, 7)
    h = batch.HostRays(rays)
    t = srv.submit_trace(ls[1], h.inp[:5], h.inp[5], 3, h.out + [h.flags], len(rays), host=True)
    srv.wait(t)
    d = batch.DeviceRays(rays)
    ref = alone(lt.REQ_TRACE, ls[1], d, len(rays), 3)
    got = (torch.stack(h.out, dim=1).numpy(), h.flags.numpy())
    assert same(got, ref)
    srv.close()


def test_admission_deadline_and_poll(lenses):
    """A budget that holds one large staged request at a time: the second
    waits (poll says not ready), a third with a 1 us deadline expires before
    it can be admitted, and everything admitted completes."""
    pres, ls = lenses
    n = 1 << 22
    # host staging (49 B/ray, arrays rounded to 16 B) + the tracer's queue (54 B/ray)
    need = 12 * n * 4 + n + (n + 64) * 54 + 256
    srv = lt.Server(mem_budget_bytes=need + 1000)
    rays = rays_for(pres[1], n, 8)
    h1, h2, h3 = batch.HostRays(rays), batch.HostRays(rays), batch.HostRays(rays)
    t1 = srv.submit_trace(ls[1], h1.inp[:5], h1.inp[5], 0, h1.out + [h1.flags], n, host=True)
    t2 = srv.submit_trace(ls[1], h2.inp[:5], h2.inp[5], 0, h2.out + [h2.flags], n, host=True)
    t3 = srv.submit_trace(ls[1], h3.inp[:5], h3.inp[5], 0, h3.out + [h3.flags], n, host=True,
                          deadline_us=1)
    st, _ = srv.poll(t2, 0)
    assert st == lt.ENOTREADY
    st, _ = srv.poll(t2, 1)
    assert st in (lt.ENOTREADY, lt.OK)
    if st == lt.ENOTREADY:
        srv.wait(t2)
    srv.wait(t1)
    st, info = srv.poll(t3, 10_000_000)
    assert st == lt.ETIMEOUT and info is not None
    s = srv.stats()
    print("admission stats", s)
    assert s["timed_out"] == 1 and s["completed"] == 2
    assert s["peak_bytes_in_flight"] <= need + 1000
    assert np.array_equal(h1.flags.numpy(), h2.flags.numpy())
    # released tickets are unknown afterwards
    st, _ = srv.poll(t1, 0)
    assert st == lt.EINVAL
    srv.close()


def test_injected_launch_failures(lenses):
    pres, ls = lenses
    srv = lt.Server(inject_fail_every=3)
    rays = rays_for(pres[0], 5000, 9)
    d = batch.DeviceRays(rays)
    ref = alone(lt.REQ_TRACE, ls[0], d, 5000, 0)
    statuses = []
    for k in range(9):
        o = batch.DeviceOut(5000)
        t = srv.submit_trace(ls[0], d.inp, d.lam, 0, o.out, 5000)
        st, info = srv.poll(t, 30_000_000)
        statuses.append(st)
        if st == lt.OK:
            torch.cuda.synchronize()
            assert same(o.numpy(), ref)
    assert statuses == [0, 0, lt.ECUDA] * 3
    assert srv.stats()["failed"] == 3
    srv.close()


def test_submit_validation(lenses):
    pres, ls = lenses
    srv = lt.Server(mem_budget_bytes=1 << 20)
    d = batch.DeviceRays(rays_for(pres[0], 64, 1))
    o = batch.DeviceOut(64)
    with pytest.raises(lt.LTError):
        srv.submit_trace(ls[0], d.inp, d.lam, ls[0].n_paths, o.out, 64)
    with pytest.raises(lt.LTError):
        srv._submit(7, d.inp, d.lam, o.out, 64, lens=ls[0])
    with pytest.raises(lt.LTError):
        srv.submit_trace(ls[0], [d.inp[0], None, d.inp[2], d.inp[3], d.inp[4]], d.lam, 0, o.out, 64)
    h = batch.HostRays(rays_for(pres[0], 1 << 16, 1))
    with pytest.raises(lt.LTError):     # staging would exceed the 1 MiB budget
        srv.submit_trace(ls[0], h.inp[:5], h.inp[5], 0, h.out + [h.flags], 1 << 16, host=True)
    t = srv.submit_trace(ls[0], d.inp, d.lam, 0, o.out, 0)
    assert srv.poll(t, 0)[0] == lt.OK
    assert srv.poll(123456789, 0)[0] == lt.EINVAL
    srv.close()


def test_concurrent_submitters(lenses):
    pres, ls = lenses
    srv = lt.Server(n_streams=4)
    errors = []

    def client(k):
        try:
            rays = rays_for(pres[k % 2], 20000 + k, 50 + k)
            d = batch.DeviceRays(rays)
            torch.cuda.synchronize()
            for rep in range(10):
                o = batch.DeviceOut(len(rays))
                torch.cuda.synchronize()
                t = srv.submit_trace(ls[k % 2], d.inp, d.lam, rep % ls[k % 2].n_paths, o.out, len(rays))
                srv.wait(t)
                if not same(o.numpy(), alone(lt.REQ_TRACE, ls[k % 2], d, len(rays),
                                             rep % ls[k % 2].n_paths)):
                    errors.append((k, rep))
        except Exception as e:     # noqa: BLE001
            errors.append(repr(e))

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert srv.stats()["completed"] == 40
    srv.close()
