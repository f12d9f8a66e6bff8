"""Training-data and schedule checks of the learned map (Sec. 5.1).

Valid-region training data: on a ghost path that few uniform draws of the
input box traverse, a map trained on uniform draws plus the valid-region
sampler's states (lt_mcmc_sample, feeding lt_mlp_train through
lt.valid_region_fit) is compared with one trained on as many uniform draws
alone, with the same schedule; both are held against the FP32 tracer on
held-out uniform rays.

Two-phase schedule of the full-transmission regressor: a first phase at
batch 32,768, then a fine-tune at batch 8,192 from learning rate 1e-6 (the
schedule Sec. 5.1 gives for it), on the backward (full transmission) map of
the reversed singlet.  The fine-tune starts from the first phase's
parameters; Adam moves every parameter by at most
lr * sqrt(10 / (1 - 0.81 / 0.999)) < 7.3 lr per step (Cauchy-Schwarz over the
moment sums with beta1 = 0.9, beta2 = 0.999; the bias corrections only
lower it for the step counts here) plus one FP32 rounding of the parameter,
so the whole phase moves none by more than steps x (7.3 lr + 2^-24 |p|)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp
from paper_2605_04017_gb300 import batch, lt, workloads as w

pytestmark = pytest.mark.gpu

WMAX10 = 0.2421


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


def xavier(seed):
    r = np.random.Generator(np.random.PCG64(seed))
    return lt.flat_params(mlp.init_params("reg", r)), lt.flat_params(mlp.init_params("cls", r))


def trace(lens, d, pid, n):
    o = batch.DeviceOut(n)
    lt.trace(lens, d.inp, d.lam, pid, o.out, n)
    torch.cuda.synchronize()
    return o.numpy()


def query(m, d, n, precision=lt.MLP_F32):
    o = batch.DeviceOut(n)
    m.query(d.inp, d.lam, o.out, n, precision)
    torch.cuda.synchronize()
    return o.numpy()


def map_error(m, lens, d, pid, n, precision=lt.MLP_F32):
    to, tf = trace(lens, d, pid, n)
    qo, qf = query(m, d, n, precision)
    tv, qv = (tf & lt.FLAG_VALID) != 0, (qf & lt.FLAG_VALID) != 0
    both = tv & qv
    e = np.hypot(qo[both, 0] - to[both, 0], qo[both, 1] - to[both, 1])
    return {"iou": float(both.sum() / max(1, (tv | qv).sum())), "agree": float((tv == qv).mean()),
            "recall": float(both.sum() / max(1, tv.sum())), "p99_mm": float(np.percentile(e, 99)),
            "rms_mm": float(np.sqrt((e ** 2).mean())), "valid": int(tv.sum())}


def test_valid_region_training_beats_uniform_on_a_sparse_ghost():
    """Of the three ghosts with the fewest valid uniform draws, the one whose
    uniform-trained map misses most of the valid region; the sampler-trained
    map of the same schedule recovers it."""
    p = w.eleven_surface_lens(oracle_accept)
    lens = lt.Lens(p)
    rho = w.eleven_rho(p)
    sm = math.tan(math.radians(10.0))
    lo, hi = [-rho, -rho, -sm, -sm, 380.0], [rho, rho, sm, sm, 780.0]
    probe = batch.DeviceRays(w.entrance_rays(1 << 18, w.SEED_BASE + 301, rho))
    frac = {}
    for pid in range(1, lens.n_paths):
        _, f = trace(lens, probe, pid, probe.n)
        frac[pid] = float(((f & lt.FLAG_VALID) != 0).mean())
    sparse = sorted(frac, key=lambda q: frac[q])[:3]
    n_u = 1 << 18
    uni = batch.DeviceRays(w.entrance_rays(n_u, w.SEED_BASE + 302, rho))
    half = batch.DeviceRays(w.entrance_rays(n_u // 2, w.SEED_BASE + 307, rho))
    held = batch.DeviceRays(w.entrance_rays(1 << 21, w.SEED_BASE + 306, rho))
    reg, cls = xavier(304)
    kw = dict(reg_steps=1500, reg_batch=8192, cls_steps=1500, cls_batch=8192, lr=1e-3, lr_decay=0.95,
              decay_every=500, seed=305)
    eu = {q: map_error(lt.Mlp.train(lens, lt.mlp_frame(q, rho, WMAX10), uni, reg, cls, **kw), lens, held, q,
                       held.n) for q in sparse}
    pid = min(sparse, key=lambda q: eu[q]["iou"])
    mc = lt.valid_region_fit(lens, pid, lo, hi, half, chains=2048, steps=64, seed=303)
    assert mc.n > n_u // 2 + 0.9 * 2048 * 64, mc.n
    frame = lt.mlp_frame(pid, rho, WMAX10)
    mu = lt.Mlp.train(lens, frame, uni, reg, cls, **kw)
    mm = lt.Mlp.train(lens, frame, mc, reg, cls, **kw)
    em = map_error(mm, lens, held, pid, held.n)
    sm_, su_ = mm.stats(), mu.stats()
    print(f"ghost path {pid} (of {sparse}): uniform valid fraction {frac[pid]:.4f}; training rays valid: "
          f"uniform {su_['n_valid']}, with sampler {sm_['n_valid']} (prefix {sm_['n_valid_uniform']}, "
          f"classifier prior shift {sm_['cls_prior_shift']:.3f})")
    print("uniform-trained", eu[pid])
    print("sampler-trained", em)
    assert su_["cls_prior_shift"] == 0.0 and su_["n_valid_uniform"] == su_["n_valid"]
    k = 1.0 + (sm_["n_valid"] - sm_["n_valid_uniform"]) / max(1, sm_["n_valid_uniform"])
    assert abs(sm_["cls_prior_shift"] - math.log(k)) < 1e-12
    assert sm_["n_valid"] > 8 * su_["n_valid"]
    assert em["iou"] > eu[pid]["iou"] + 0.05, (eu[pid], em)
    assert em["recall"] > eu[pid]["recall"], (eu[pid], em)
    assert em["p99_mm"] < 1.1 * eu[pid]["p99_mm"], (eu[pid], em)


def test_training_is_reproducible():
    """The valid list is built in ray order and every reduction has a fixed
    order, so two trainings on the same inputs give the same bits."""
    p = w.singlet_lens()
    lens = lt.Lens(p)
    fit = batch.DeviceRays(w.entrance_rays(100003, 51, 12.0))
    reg, cls = xavier(52)
    runs = [lt.Mlp.train(lens, lt.mlp_frame(0, 12.0, WMAX10), fit, reg, cls, reg_steps=200, reg_batch=8192,
                         cls_steps=100, cls_batch=8192, lr=1e-3, seed=53) for _ in range(2)]
    (r0, c0), (r1, c1) = runs[0].params(), runs[1].params()
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1)
    s0, s1 = runs[0].stats(), runs[1].stats()
    assert s0["t_mean"] == s1["t_mean"] and s0["t_std"] == s1["t_std"] and s0["n_valid"] == s1["n_valid"]


def test_backward_map_two_phase_fine_tune():
    p = w.singlet_lens()
    fwd = lt.Lens(p)
    zi = fwd.paraxial(w.LAMBDA_D_NM)[2]
    back = fwd.reversed(zi, 0.0)
    rho = 9.0
    wmax = 0.3544        # |d_xy| of a direction with |theta_x|, |theta_y| <= 15 deg is <= 0.35435
    frame = lt.mlp_frame(0, rho, wmax)
    fit = batch.DeviceRays(w.entrance_rays(1 << 18, 41, rho, 15.0))
    reg0, cls0 = xavier(42)
    a = lt.Mlp.train(back, frame, fit, reg0, cls0, reg_steps=2000, reg_batch=32768, cls_steps=600,
                     cls_batch=8192, lr=1e-3, lr_decay=0.95, decay_every=500, seed=43)
    reg_a, cls_a = a.params()
    # fine-tune phase alone, from the first phase's parameters
    F, ft_lr = 1000, 1e-6
    b = lt.Mlp.train(back, frame, fit, reg_a, cls_a, reg_steps=0, cls_steps=0, ft_steps=F, ft_batch=8192,
                     ft_lr=ft_lr, lr_decay=0.95, decay_every=500, seed=43)
    reg_b, cls_b = b.params()
    assert np.array_equal(cls_b, cls_a)
    dp = np.abs(reg_b.astype(np.float64) - reg_a)
    bound = F * (7.3 * ft_lr + 2.0 ** -24 * np.abs(reg_a.astype(np.float64)).max())
    assert 0 < dp.max() <= bound, (dp.max(), bound)
    assert (dp > 0).mean() > 0.5
    # a zero learning rate leaves every parameter bit-for-bit
    z = lt.Mlp.train(back, frame, fit, reg_a, cls_a, reg_steps=0, cls_steps=0, ft_steps=50, ft_batch=8192,
                     ft_lr=0.0, seed=45)
    assert np.array_equal(z.params()[0], reg_a)
    # the full schedule in one call, and what the fine-tune does to the map
    c = lt.Mlp.train(back, frame, fit, reg0, cls0, reg_steps=2000, reg_batch=32768, cls_steps=600,
                     cls_batch=8192, lr=1e-3, lr_decay=0.95, decay_every=500, ft_steps=F, ft_batch=8192,
                     ft_lr=ft_lr, seed=43)
    # training is reproducible, so the one-call schedule is the first phase
    # followed by the same fine-tune, bit for bit
    assert np.array_equal(c.params()[0], reg_b) and np.array_equal(c.params()[1], cls_a)
    held = batch.DeviceRays(w.entrance_rays(1 << 18, 46, rho, 15.0))
    ea, eb, ec = (map_error(m, back, held, 0, held.n) for m in (a, b, c))
    print("backward map: first phase", ea, "fine-tuned", eb, "two phases in one call", ec)
    assert eb["rms_mm"] <= 1.01 * ea["rms_mm"]
    assert ec["rms_mm"] <= 1.5 * ea["rms_mm"] and ec["recall"] > 0.95
