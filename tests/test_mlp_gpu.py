"""GPU checks of the learned map (paper Sec. 4.2 classifier/regressor, Sec. 5.1
training and inference) against the oracle's FP64 networks (oracle/mlp.py).

Tolerances.  Gradients: the GPU computes forward/backward in FP32 with FP32
per-block sums of 128 rays and an FP64 sum over blocks; relative to the
largest gradient entry that is ~1e-6, the test allows 1e-4.  Queries are
compared ray by ray (tests/mlp_check.py): FP32 to 3e-5 of each output's
standard deviation plus two FP32 ulps, BF16 / FP16 to twice a first-order
bound of the half-precision rounding of the six layers, computed per ray
from the oracle's activations."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp
from paper_2605_04017_gb300 import batch, lt, workloads as w

from mlp_check import check_query

pytestmark = pytest.mark.gpu

RHO = 12.0
WMAX = 0.2421    # |d_xy| of a direction with |theta_x|, |theta_y| <= 10 deg is <= 0.2420


def frame(path_id=0):
    return lt.mlp_frame(path_id, RHO, WMAX)


def init(seed):
    r = np.random.Generator(np.random.PCG64(seed))
    return mlp.init_params("reg", r), mlp.init_params("cls", r)


def as64(flat, kind):
    return lt.unflat_params(flat, mlp.layer_sizes(kind))


def targets(L, rays):
    out, v, _, _ = L.trace(rays)
    arrs = [a.astype(np.float64) for a in rays.arrays()]
    r, dxr, dyr, lam, phi, mir = mlp.reduce_frame(*arrs)
    return mlp.reduce_outputs(out, phi, mir), v == 1


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.fixture(scope="module")
def singlet():
    p = w.singlet_lens()
    return p, lt.Lens(p), oracle.Lens(p)


@pytest.fixture(scope="module")
def tstats(singlet):
    p, lens, ol = singlet
    T, valid = targets(ol, w.singlet_rays(20000))
    return mlp.standardise(T[valid])


def test_features_match_oracle(singlet, tstats):
    p, lens, ol = singlet
    reg, cls = init(1)
    m = lt.Mlp.create(lens, frame(), lt.flat_params(reg), lt.flat_params(cls), *tstats)
    rays = w.singlet_rays(5000)
    d = batch.DeviceRays(rays)
    X = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    m.features(d.inp, d.lam, X, len(rays))
    torch.cuda.synchronize()
    Xo, _, _ = mlp.features(rays.arrays(), RHO, WMAX)
    assert np.abs(X.cpu().numpy() - Xo).max() < 2e-6


@pytest.mark.parametrize("net,B", [(0, 1000), (0, 128), (1, 777)])
def test_gradients_match_oracle(singlet, tstats, net, B):
    p, lens, ol = singlet
    reg, cls = init(2)
    reg_f, cls_f = lt.flat_params(reg), lt.flat_params(cls)
    m = lt.Mlp.create(lens, frame(), reg_f, cls_f, *tstats)
    rays = w.singlet_rays(4 * B)
    T, valid = targets(ol, rays)
    X, _, _ = mlp.features(rays.arrays(), RHO, WMAX)
    X32 = X.astype(np.float32)
    t_mean, t_std = tstats
    if net == 0:
        sel = np.nonzero(valid)[0][:B]
        Xb = X32[sel]
        Tb = ((T[sel] - t_mean) / t_std).astype(np.float32)
        params = as64(reg_f, "reg")
        acts = mlp.forward(params, Xb.astype(np.float64))
        loss, dout = mlp.regressor_loss(acts[-1], Tb.astype(np.float64), t_std[2:5], t_mean[2:5])
        g_or = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in
                               mlp.backward(params, acts, dout)])
        g, l = m.grad(0, dev(Xb), dev(Tb), len(sel))
    else:
        Xb = X32[:B]
        yb = valid[:B].astype(np.float32)
        params = as64(cls_f, "cls")
        acts = mlp.forward(params, Xb.astype(np.float64))
        loss, dout = mlp.classifier_loss(acts[-1], yb.astype(np.float64))
        g_or = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in
                               mlp.backward(params, acts, dout)])
        g, l = m.grad(1, dev(Xb), dev(yb), B)
    rel = np.abs(g - g_or).max() / np.abs(g_or).max()
    print("grad", net, B, "rel err", rel, "loss", l, loss)
    assert rel < 1e-4
    assert l == pytest.approx(loss, rel=1e-5)


def run_query(m, rays, precision):
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(len(rays))
    m.query(d.inp, d.lam, o.out, len(rays), precision)
    torch.cuda.synchronize()
    return o.numpy()


def test_query_f32_matches_oracle_forward(singlet, tstats):
    p, lens, ol = singlet
    reg, cls = init(3)
    reg_f, cls_f = lt.flat_params(reg), lt.flat_params(cls)
    t_mean, t_std = tstats
    m = lt.Mlp.create(lens, frame(), reg_f, cls_f, t_mean, t_std)
    rays = w.singlet_rays(20000)
    out, flags = run_query(m, rays, lt.MLP_F32)
    rep = check_query(out, flags, as64(reg_f, "reg"), as64(cls_f, "cls"), rays, RHO, WMAX, t_mean, t_std,
                      lt.MLP_F32, "singlet, random networks")
    assert rep["decided"] > 0.99


@pytest.mark.parametrize("precision", [lt.MLP_BF16, lt.MLP_F16])
def test_query_half_precision_matches_oracle_forward(singlet, tstats, precision):
    """The tensor-core queries of random networks, ray by ray, within the
    half-precision rounding bound."""
    p, lens, ol = singlet
    reg, cls = init(4)
    reg_f, cls_f = lt.flat_params(reg), lt.flat_params(cls)
    t_mean, t_std = tstats
    m = lt.Mlp.create(lens, frame(), reg_f, cls_f, t_mean, t_std)
    rays = w.singlet_rays(20000)
    out, flags = run_query(m, rays, precision)
    rep = check_query(out, flags, as64(reg_f, "reg"), as64(cls_f, "cls"), rays, RHO, WMAX, t_mean, t_std,
                      precision, "singlet, random networks")
    print("precision", precision, rep)
    assert rep["decided"] > 0.75 and rep["compared"] > 1000


def test_bad_precision_is_rejected(singlet, tstats):
    p, lens, ol = singlet
    reg, cls = init(5)
    m = lt.Mlp.create(lens, frame(), lt.flat_params(reg), lt.flat_params(cls), *tstats)
    rays = w.singlet_rays(8)
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(8)
    with pytest.raises(lt.LTError):
        m.query(d.inp, d.lam, o.out, 8, 17)


@pytest.fixture(scope="module")
def trained(singlet):
    p, lens, ol = singlet
    fit = w.entrance_rays(1 << 19, w.SEED_BASE + 101, RHO)
    reg, cls = init(6)
    m = lt.Mlp.train(lens, frame(), batch.DeviceRays(fit), lt.flat_params(reg), lt.flat_params(cls),
                     reg_steps=6000, reg_batch=8192, cls_steps=4000, cls_batch=8192, lr=1e-3,
                     lr_decay=0.95, decay_every=500, seed=11)
    return m, reg, cls


def test_training_learns(singlet, trained):
    p, lens, ol = singlet
    m, reg0, cls0 = trained
    st = m.stats()
    print("training", st)
    assert st["n_train"] == 1 << 19 and 0.5 < st["n_valid"] / st["n_train"] < 0.9
    # initial loss of the same networks, computed by the oracle
    rays = w.entrance_rays(20000, 77, RHO)
    T, valid = targets(ol, rays)
    X, _, _ = mlp.features(rays.arrays(), RHO, WMAX)
    tm, ts = np.array(st["t_mean"]), np.array(st["t_std"])
    Tn = (T[valid] - tm) / ts
    l0, _ = mlp.regressor_loss(mlp.forward(reg0, X[valid])[-1], Tn, ts[2:5], tm[2:5])
    reg_f, cls_f = m.params()
    l1, _ = mlp.regressor_loss(mlp.forward(as64(reg_f, "reg"), X[valid])[-1], Tn, ts[2:5], tm[2:5])
    print("regressor loss", l0, "->", l1, "(GPU training tail", st["reg_loss"], ")")
    assert l1 < 0.05 * l0
    acc = ((mlp.forward(as64(cls_f, "cls"), X)[-1][:, 0] > 0) == valid).mean()
    print("classifier accuracy", acc)
    assert acc > 0.95


def test_learned_map_gain(singlet, trained):
    """What the trained networks gain: the classifier removes occluded rays
    that the regressor alone would send to the sensor (paper Fig. 6), and the
    learned map answers every ray without falling back to the tracer."""
    p, lens, ol = singlet
    m, _, _ = trained
    rays = w.singlet_rays()
    ex, ev, _, _ = ol.trace(rays)
    truth = ev == 1
    o_c, f_c = run_query(m, rays, lt.MLP_F32)
    o_n, f_n = run_query(m, rays, lt.MLP_F32_NOCLS)
    fv_c = (((f_c & 1) != 0) & ~truth).mean()
    fv_n = (((f_n & 1) != 0) & ~truth).mean()
    I_true = ex[truth, 5].sum()
    print("false-valid with / without classifier", fv_c, fv_n,
          "exposure ratio", o_c[:, 5].sum() / I_true, o_n[:, 5].sum() / I_true)
    invalid = (~truth).mean()
    assert fv_n > 0.9 * invalid and fv_c < 0.2 * invalid
    assert abs(o_c[:, 5].sum() / I_true - 1) < 0.05 and o_n[:, 5].sum() / I_true > 1.05
    # the learned map never calls the tracer; the table map of the same lens does
    sm = math.tan(math.radians(10))
    g = lt.Map.build(lens, 0, [32, 32, 32, 32, 8], [-RHO, -RHO, -sm, -sm, 380], [RHO, RHO, sm, sm, 780],
                     fit=batch.DeviceRays(rays))
    d = batch.DeviceRays(rays)
    ot = batch.DeviceOut(len(rays))
    g.query(d.inp, d.lam, ot.out, len(rays))
    torch.cuda.synchronize()
    _, ft = ot.numpy()
    assert ((f_c & lt.FLAG_TRACED) == 0).all()
    print("table-map fallback fraction", ((ft & lt.FLAG_TRACED) != 0).mean())
    # position error of the learned map on rays both call valid (reported)
    both = ((f_c & 1) != 0) & truth
    e = np.hypot(o_c[both, 0] - ex[both, 0], o_c[both, 1] - ex[both, 1])
    print("learned map position error rms / p99 (mm)", np.sqrt((e ** 2).mean()), np.percentile(e, 99))


@pytest.fixture(scope="module")
def precision_batch():
    return w.precision_rays()


@pytest.mark.parametrize("precision", [lt.MLP_F32, lt.MLP_BF16, lt.MLP_F16])
def test_full_size_precision_queries_sampled(singlet, trained, precision_batch, precision):
    """The precision workload as the bench runs it: the trained networks
    answer all 16,777,216 rays in one launch; 4,098 rays spread over the batch
    (the first and last included) are checked against the oracle's forward
    ray by ray, with the tolerances of the small tests."""
    p, lens, ol = singlet
    m, _, _ = trained
    rays = precision_batch
    n = len(rays)
    assert n == 16777216
    out, flags = run_query(m, rays, precision)
    rng = np.random.Generator(np.random.PCG64(91))
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 4096)]))
    sample = rays.subset(idx)
    out, flags = out[idx], flags[idx]
    st = m.stats()
    t_mean, t_std = np.array(st["t_mean"]), np.array(st["t_std"])
    reg_f, cls_f = m.params()
    rep = check_query(out, flags, as64(reg_f, "reg"), as64(cls_f, "cls"), sample, RHO, WMAX, t_mean, t_std,
                      precision, "singlet, trained, 16.7 M rays")
    print("full-size precision", precision, rep)
