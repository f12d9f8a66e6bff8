"""The tracer's hand-written FP32 reciprocal and square root (lt_tracer_math)
against correctly rounded results: numpy's float32 division and square root
are IEEE correctly rounded, as are CUDA's __frcp_rn and __fsqrt_rn.  The
reciprocal is the hardware approximation plus one Newton-Raphson step, the
square root the hardware reciprocal square root plus one Newton step; both
are held to 1 ulp over every binade they are used on."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_04017_gb300 import lt

pytestmark = pytest.mark.gpu


def ulps(a, b):
    """Distance in units in the last place between float32 arrays of one sign."""
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def run(x):
    d = torch.from_numpy(x).cuda()
    r = torch.empty_like(d)
    s = torch.empty_like(d)
    lt.tracer_math(d, r, s, len(x))
    torch.cuda.synchronize()
    return r.cpu().numpy(), s.cpu().numpy()


def sample(n, lo_exp, hi_exp, seed):
    """Floats spread log-uniformly over [2^lo_exp, 2^hi_exp), with the special
    cases of the tracer's ranges (powers of two, their neighbours, 1.5)."""
    g = np.random.default_rng(seed)
    m = g.uniform(1.0, 2.0, n).astype(np.float32)
    e = g.integers(lo_exp, hi_exp, n)
    x = np.ldexp(m, e).astype(np.float32)
    p2 = np.ldexp(np.float32(1.0), np.arange(lo_exp, hi_exp)).astype(np.float32)
    extra = np.concatenate([p2, np.nextafter(p2, np.float32(0)), np.nextafter(p2, np.float32(np.inf)),
                            np.float32([1.0, 1.5, 1.0000001, 0.9999999])])
    return np.concatenate([x, extra]).astype(np.float32)


def test_reciprocal_within_one_ulp():
    # 1/x normal for |x| in [2^-125, 2^125]; both signs
    x = sample(1 << 20, -125, 125, 1)
    x = np.concatenate([x, -x])
    r, _ = run(x)
    ref = (np.float32(1.0) / x).astype(np.float32)
    u = ulps(r, ref)
    print("rcp: max ulp", int(u.max()), "exact", float((u == 0).mean()))
    assert u.max() <= 1
    assert (u == 0).mean() > 0.9


def test_square_root_within_one_ulp():
    x = sample(1 << 20, -126, 127, 2)
    _, s = run(x)
    ref = np.sqrt(x).astype(np.float32)
    u = ulps(s, ref)
    print("sqrt: max ulp", int(u.max()), "exact", float((u == 0).mean()))
    assert u.max() <= 1
    # non-positive inputs give 0, as the tracer's tests of a discriminant need
    _, z = run(np.float32([0.0, -0.0, -1.0, -3e-38]))
    assert np.all(z == 0.0)


def test_rejects_null_arrays():
    with pytest.raises(lt.LTError):
        lt.tracer_math(None, None, None, 4)
    lt.tracer_math(None, None, None, 0)
