"""Pins for the oracle's learned map (oracle/mlp.py): gradients against
central finite differences, closed-form special cases, the symmetry frame
against direct rotation/mirroring, and Adam's first step in closed form."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2605_04017_gb300 import workloads as w


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def fd_check(params, loss_fn, h=1e-5, n_probe=60, seed=1):
    """Largest |central difference - hand-written gradient| over random
    entries, relative to the largest gradient entry."""
    acts = mlp.forward(params, loss_fn.X)
    loss, dout = loss_fn(acts[-1])
    grads = mlp.backward(params, acts, dout)
    gmax = max(float(np.abs(g).max()) for gg in grads for g in gg)
    r = rng(seed)
    worst = 0.0
    for _ in range(n_probe):
        li = int(r.integers(len(params)))
        which = int(r.integers(2))
        P = params[li][which]
        idx = tuple(int(r.integers(s)) for s in P.shape)
        old = P[idx]
        P[idx] = old + h
        lp = loss_fn(mlp.forward(params, loss_fn.X)[-1])[0]
        P[idx] = old - h
        lm = loss_fn(mlp.forward(params, loss_fn.X)[-1])[0]
        P[idx] = old
        fd = (lp - lm) / (2 * h)
        g = grads[li][which][idx]
        worst = max(worst, abs(fd - g) / gmax)
    return worst


class RegLoss:
    def __init__(self, X, T, scale, mean):
        self.X, self.T, self.scale, self.mean = X, T, scale, mean

    def __call__(self, pred):
        return mlp.regressor_loss(pred, self.T, self.scale, self.mean)


class ClsLoss:
    def __init__(self, X, y):
        self.X, self.y = X, y

    def __call__(self, logit):
        return mlp.classifier_loss(logit, self.y)


def test_regressor_gradient_matches_finite_differences():
    r = rng(3)
    params = mlp.init_params("reg", r)
    X = r.uniform(-1, 1, size=(64, 4))
    T = r.normal(size=(64, 6))
    loss = RegLoss(X, T, np.array([0.1, 0.2, 0.05]), np.array([0.0, 0.1, 0.9]))
    assert fd_check(params, loss) < 1e-7


def test_classifier_gradient_matches_finite_differences():
    r = rng(4)
    params = mlp.init_params("cls", r)
    X = r.uniform(-1, 1, size=(64, 4))
    y = (r.uniform(size=64) < 0.4).astype(float)
    assert fd_check(params, ClsLoss(X, y)) < 1e-7


def test_bce_gradient_is_sigmoid_minus_label():
    z = np.array([[-3.0], [0.0], [2.5], [40.0], [-40.0]])
    y = np.array([0, 1, 1, 0, 1.0])
    loss, g = mlp.classifier_loss(z, y)
    sig = 1 / (1 + np.exp(-z[:, 0]))
    assert np.allclose(g[:, 0] * len(y), sig - y, atol=1e-15)
    # large |z| stays finite: BCE(40, 0) = 40, BCE(-40, 1) = 40
    assert math.isfinite(loss)
    assert loss == pytest.approx((math.log1p(math.exp(-3)) + math.log(2) +
                                  math.log1p(math.exp(-2.5)) + 40 + 40) / 5, rel=1e-12)


def test_forward_closed_forms():
    # zero weights: the output is the last bias
    params = [(np.zeros((32, 4)), np.zeros(32)), (np.zeros((1, 32)), np.array([0.7]))]
    assert np.allclose(mlp.forward(params, np.ones((3, 4)))[-1], 0.7)
    # one active unit: y = w2 * tanh(w1 . x + b1) + b2
    W1 = np.zeros((32, 4))
    W1[5] = [0.3, -0.2, 0.1, 0.4]
    b1 = np.zeros(32)
    b1[5] = 0.05
    W2 = np.zeros((1, 32))
    W2[0, 5] = 1.7
    x = np.array([[0.2, 0.9, -0.4, 0.6]])
    y = mlp.forward([(W1, b1), (W2, np.array([-0.1]))], x)[-1][0, 0]
    assert y == pytest.approx(1.7 * math.tanh(0.06 - 0.18 - 0.04 + 0.24 + 0.05) - 0.1, rel=1e-15)


def test_regressor_loss_closed_form():
    pred = np.array([[1.0, 2.0, 0.0, 0.0, 1.0, 0.5]])
    targ = np.array([[0.0, 0.0, 0.0, 1.0, 0.0, 0.0]])
    loss, _ = mlp.regressor_loss(pred, targ, np.ones(3), np.zeros(3))
    # position 0.5*(1+4), I 0.25, perpendicular directions: 1 - cos = 1
    assert loss == pytest.approx(2.5 + 0.25 + 1.0, rel=1e-15)


def test_adam_first_step_closed_form():
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -7.0]]), np.array([1e-3]))]
    opt = mlp.Adam(params, lr=1e-2)
    new = opt.step(params, grads)
    # bias-corrected first step is lr * g / (|g| + eps) = lr * sign(g) (to eps/|g|)
    assert np.allclose(new[0][0], [[1.0 - 1e-2, -2.0 + 1e-2]], atol=1e-9)
    assert new[0][1][0] == pytest.approx(0.5 - 1e-2 * 1e-3 / (1e-3 + 1e-8), rel=1e-12)


def test_lr_schedule():
    assert mlp.lr_at(0) == 1e-4
    assert mlp.lr_at(9999) == 1e-4
    assert mlp.lr_at(10000) == pytest.approx(0.95e-4)
    assert mlp.lr_at(25000) == pytest.approx(1e-4 * 0.95 ** 2)


def test_reduced_frame_round_trip_and_invariance():
    rays = w.singlet_rays(500)
    arrs = [a.astype(np.float64) for a in rays.arrays()]
    r, dxr, dyr, lam, phi, mir = mlp.reduce_frame(*arrs)
    assert np.all(dyr >= 0) and np.all(r >= 0)
    # rotating the input ray about the axis leaves the reduced coordinates unchanged
    a = 0.83
    c, s = math.cos(a), math.sin(a)
    rot = [c * arrs[0] - s * arrs[1], s * arrs[0] + c * arrs[1], c * arrs[2] - s * arrs[3],
           s * arrs[2] + c * arrs[3], arrs[4], arrs[5]]
    r2, dxr2, dyr2, _, _, _ = mlp.reduce_frame(*rot)
    assert np.allclose(r2, r) and np.allclose(dxr2, dxr, atol=1e-14) and np.allclose(dyr2, dyr, atol=1e-14)
    # mirroring y does too
    mir_ray = [arrs[0], -arrs[1], arrs[2], -arrs[3], arrs[4], arrs[5]]
    r3, dxr3, dyr3, _, _, _ = mlp.reduce_frame(*mir_ray)
    assert np.allclose(dxr3, dxr, atol=1e-14) and np.allclose(dyr3, dyr, atol=1e-14)
    # outputs: reduce then unreduce is the identity
    out = np.random.default_rng(2).normal(size=(500, 6))
    back = mlp.unreduce_outputs(mlp.reduce_outputs(out, phi, mir), phi, mir)
    assert np.allclose(back, out, atol=1e-13)


def test_reduced_frame_matches_oracle_equivariance():
    """The traced map is itself equivariant (Eq. 10): traced outputs expressed
    in the reduced frame depend only on the reduced inputs."""
    p = w.singlet_lens()
    L = oracle.Lens(p)
    rays = w.singlet_rays(300)
    out, v, _, _ = L.trace(rays)
    arrs = [a.astype(np.float64) for a in rays.arrays()]
    r, dxr, dyr, lam, phi, mir = mlp.reduce_frame(*arrs)
    red = mlp.reduce_outputs(out, phi, mir)
    # the same ray placed directly in the reduced frame
    nrm = np.sqrt(dxr ** 2 + dyr ** 2)
    dz = np.sqrt(1 - nrm ** 2)
    f = np.float64
    for k in np.nonzero(v == 1)[0][:100]:
        vv, o2, _, _ = L.trace_one(r[k], 0.0, dxr[k], dyr[k], dz[k], lam[k])
        assert vv == 1
        assert np.allclose(o2, red[k], atol=2e-5)


def test_query_masks_invalid():
    r = rng(7)
    cls = mlp.init_params("cls", r)
    reg = mlp.init_params("reg", r)
    rays = w.singlet_rays(200)
    out, valid, logit = mlp.query(cls, reg, rays, 12.0, 0.25, np.zeros(6), np.ones(6))
    assert np.all(out[~valid] == 0.0)
    assert np.allclose(np.linalg.norm(out[valid, 2:5], axis=1), 1.0)


def test_lambert_tanh_error_bound_and_series():
    x = np.linspace(-20, 20, 400001)
    err = np.abs(mlp.tanh_lambert(x) - np.tanh(x))
    assert err.max() < 1.9e-6
    # the 9/10 truncation agrees with the Taylor series of tanh to high order at small x
    s = np.array([1e-3, 0.05, 0.1])
    taylor = s - s ** 3 / 3 + 2 * s ** 5 / 15 - 17 * s ** 7 / 315 + 62 * s ** 9 / 2835
    assert np.allclose(mlp.tanh_lambert(s), taylor, rtol=0, atol=1e-12)
    assert np.allclose(mlp.tanh_lambert(-x), -mlp.tanh_lambert(x))
    assert mlp.tanh_lambert(np.array([7.0]))[0] == 1.0
