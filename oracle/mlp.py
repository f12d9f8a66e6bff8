"""ORACLE (test infrastructure only): the learned lens transport map, FP64 numpy.

What it computes, from the paper:
  - domain reduction by the lens symmetry (Sec. 4.1, Eq. 10): rotate the
    entrance ray about the axis so its point lies on +x (p -> (r, 0)), then
    mirror y -> -y if the rotated direction has d_y < 0; the network sees
    (r, d_x', d_y' >= 0, lambda) and its outputs are mirrored and rotated back;
    the throughput is invariant;
  - per path, a binary classifier g(x) and a regressor f(x) used only where
    g(x) = 1 (Sec. 4.2, Eq. 11);
  - compact MLPs, width 32, tanh hidden layers, linear output; regressor with
    five hidden layers, classifier with two (Sec. 5.1);
  - losses: mean squared error on exit position and throughput, cosine
    similarity on exit direction (regressor); binary cross-entropy
    (classifier) (Sec. 5.1);
  - optimisation: learning rate 1e-4 decaying by 0.95 every 10,000 batches
    (Sec. 5.1).  The optimiser is not named; Adam (beta1 0.9, beta2 0.999,
    eps 1e-8) is used, with Xavier-uniform weights and zero biases.
Readings where the paper is silent: inputs normalised to [-1, 1] over the
map box; regressor targets are the reduced-frame exit (x', y'), direction
(3 components) and I, each standardised by the training set's mean and
standard deviation; the regressor loss per ray is
  ((x^ - x)^2 + (y^ - y)^2) / 2 + (I^ - I)^2 + (1 - cos(d^, d))
in standardised units (cosine on the de-standardised direction), averaged
over the batch.

Everything here is a plain restatement: matrix products are numpy's, the
backward pass is the chain rule written out layer by layer.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

WIDTH = 32
REG_HIDDEN = 5
CLS_HIDDEN = 2
N_IN = 4
N_REG_OUT = 6


# ----------------------------------------------------------------------------- frame

def reduce_frame(x, y, dx, dy, dz, lam):
    """Symmetry-reduced entrance ray: returns (r, dxr, dyr, lam, phi, mirror)
    with dyr >= 0; mirror = -1 where the y axis was flipped, else +1."""
    x, y, dx, dy, dz, lam = [np.asarray(a, np.float64) for a in (x, y, dx, dy, dz, lam)]
    nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
    dx, dy = dx / nrm, dy / nrm
    r = np.hypot(x, y)
    phi = np.arctan2(y, x)
    c, s = np.cos(phi), np.sin(phi)
    dxr = c * dx + s * dy
    dyr = -s * dx + c * dy
    mirror = np.where(dyr < 0.0, -1.0, 1.0)
    return r, dxr, dyr * mirror, lam, phi, mirror


def reduce_outputs(out6, phi, mirror):
    """Exit ray (x, y, dx, dy, dz, I) -> reduced frame of its entrance ray."""
    c, s = np.cos(phi), np.sin(phi)
    o = np.array(out6, np.float64, copy=True)
    xr = c * out6[:, 0] + s * out6[:, 1]
    yr = -s * out6[:, 0] + c * out6[:, 1]
    dxr = c * out6[:, 2] + s * out6[:, 3]
    dyr = -s * out6[:, 2] + c * out6[:, 3]
    o[:, 0], o[:, 1] = xr, yr * mirror
    o[:, 2], o[:, 3] = dxr, dyr * mirror
    return o


def unreduce_outputs(red6, phi, mirror):
    """Inverse of reduce_outputs."""
    c, s = np.cos(phi), np.sin(phi)
    o = np.array(red6, np.float64, copy=True)
    xr, yr = red6[:, 0], red6[:, 1] * mirror
    dxr, dyr = red6[:, 2], red6[:, 3] * mirror
    o[:, 0] = c * xr - s * yr
    o[:, 1] = s * xr + c * yr
    o[:, 2] = c * dxr - s * dyr
    o[:, 3] = s * dxr + c * dyr
    return o


def features(rays, rho, wmax, lam_lo=380.0, lam_hi=780.0):
    """Network inputs in [-1, 1]: r over [0, rho], d_x' over [-wmax, wmax],
    d_y' over [0, wmax], lambda over [lam_lo, lam_hi].  Returns (X, phi, mirror)."""
    r, dxr, dyr, lam, phi, mirror = reduce_frame(*rays)
    X = np.stack([2.0 * r / rho - 1.0, dxr / wmax, 2.0 * dyr / wmax - 1.0,
                  2.0 * (lam - lam_lo) / (lam_hi - lam_lo) - 1.0], axis=1)
    return X, phi, mirror


# ----------------------------------------------------------------------------- networks

def layer_sizes(kind: str) -> List[int]:
    if kind == "reg":
        return [N_IN] + [WIDTH] * REG_HIDDEN + [N_REG_OUT]
    if kind == "cls":
        return [N_IN] + [WIDTH] * CLS_HIDDEN + [1]
    raise ValueError(kind)


def init_params(kind: str, rng: np.random.Generator):
    """Xavier-uniform weights W[l] of shape (out, in), zero biases."""
    sz = layer_sizes(kind)
    params = []
    for a, b in zip(sz[:-1], sz[1:]):
        lim = math.sqrt(6.0 / (a + b))
        params.append((rng.uniform(-lim, lim, size=(b, a)), np.zeros(b)))
    return params


def forward(params, X):
    """Returns the list of layer outputs: a[0] = X, a[l] = tanh(W a + b) for
    hidden layers, the last entry linear."""
    acts = [np.asarray(X, np.float64)]
    for li, (W, b) in enumerate(params):
        z = acts[-1] @ W.T + b
        acts.append(z if li == len(params) - 1 else np.tanh(z))
    return acts


def backward(params, acts, dout):
    """Gradients of a loss with d loss / d output = dout (batch x out)."""
    grads = [None] * len(params)
    delta = dout
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        grads[li] = (delta.T @ acts[li], delta.sum(axis=0))
        if li > 0:
            delta = (delta @ W) * (1.0 - acts[li] ** 2)     # tanh' = 1 - tanh^2
    return grads


# ----------------------------------------------------------------------------- losses

def regressor_loss(pred, target, dir_scale, dir_mean):
    """Loss and d loss / d pred for standardised predictions and targets
    (columns x', y', dx', dy', dz', I).  The direction enters the cosine
    de-standardised: d = mean + scale * z."""
    B = pred.shape[0]
    ep = pred[:, 0:2] - target[:, 0:2]
    ei = pred[:, 5] - target[:, 5]
    dp = dir_mean + dir_scale * pred[:, 2:5]
    dt = dir_mean + dir_scale * target[:, 2:5]
    npd = np.linalg.norm(dp, axis=1)
    ntd = np.linalg.norm(dt, axis=1)
    cos = np.sum(dp * dt, axis=1) / (npd * ntd)
    loss = np.mean(0.5 * np.sum(ep ** 2, axis=1) + ei ** 2 + (1.0 - cos))
    g = np.zeros_like(pred)
    g[:, 0:2] = ep / B
    g[:, 5] = 2.0 * ei / B
    # d(-cos)/d dp = -(dt/(|dp||dt|) - cos * dp/|dp|^2)
    dcos = dt / (npd * ntd)[:, None] - cos[:, None] * dp / (npd ** 2)[:, None]
    g[:, 2:5] = -dcos * dir_scale / B
    return loss, g


def classifier_loss(logit, label):
    """Binary cross-entropy on logits (mean) and its gradient."""
    z = logit[:, 0]
    y = np.asarray(label, np.float64)
    loss = np.mean(np.maximum(z, 0.0) - y * z + np.log1p(np.exp(-np.abs(z))))
    sig = 1.0 / (1.0 + np.exp(-z))
    g = ((sig - y) / len(z))[:, None]
    return loss, g


# ----------------------------------------------------------------------------- optimiser

class Adam:
    def __init__(self, params, lr=1e-4, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads, lr=None):
        lr = self.lr if lr is None else lr
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        new = []
        for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            out = []
            for k, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[li][k] + (1.0 - self.b1) * g
                v = self.b2 * self.v[li][k] + (1.0 - self.b2) * g * g
                self.m[li] = (m, self.m[li][1]) if k == 0 else (self.m[li][0], m)
                self.v[li] = (v, self.v[li][1]) if k == 0 else (self.v[li][0], v)
                out.append(p - lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            new.append((out[0], out[1]))
        return new


def lr_at(step, lr0=1e-4, decay=0.95, every=10000):
    """Exponential schedule of Sec. 5.1: lr0 * decay^(floor(step / every))."""
    return lr0 * decay ** (step // every)


# ----------------------------------------------------------------------------- map

def standardise(T):
    mean = T.mean(axis=0)
    std = T.std(axis=0)
    std[std == 0.0] = 1.0
    return mean, std


def query(cls_params, reg_params, rays, rho, wmax, t_mean, t_std, lam_lo=380.0, lam_hi=780.0):
    """Learned-map query (Eq. 11): outputs (n x 6) and validity (logit > 0)."""
    X, phi, mirror = features(rays.arrays() if hasattr(rays, "arrays") else rays, rho, wmax,
                              lam_lo, lam_hi)
    logit = forward(cls_params, X)[-1][:, 0]
    valid = logit > 0.0
    z = forward(reg_params, X)[-1]
    red = t_mean + t_std * z
    d = red[:, 2:5]
    red[:, 2:5] = d / np.linalg.norm(d, axis=1, keepdims=True)
    out = unreduce_outputs(red, phi, mirror)
    out[~valid] = 0.0
    return out, valid, logit


# ----------------------------------------------------------------------------- inference tanh

# Sec. 5.1: inference replaces tanh by a rational function.  Reading: the
# truncation of Lambert's continued fraction
#   tanh x = x / (1 + x^2 / (3 + x^2 / (5 + x^2 / (7 + ...))))
# after the 19 term, i.e. the 9/10 Pade approximant, clamped to +-1 for
# |x| >= 6.95 (where the truncation error and 1 - tanh cross).
_LAMBERT_NUM = [654729075.0, 91891800.0, 2837835.0, 25740.0, 55.0]
_LAMBERT_DEN = [654729075.0, 310134825.0, 18918900.0, 315315.0, 1485.0, 1.0]


def tanh_lambert(x):
    x = np.asarray(x, np.float64)
    x2 = x * x
    num = np.zeros_like(x)
    for c in reversed(_LAMBERT_NUM):
        num = num * x2 + c
    den = np.zeros_like(x)
    for c in reversed(_LAMBERT_DEN):
        den = den * x2 + c
    y = x * num / den
    return np.where(np.abs(x) >= 6.95, np.sign(x), y)


def forward_with(params, X, act):
    """forward() with a given hidden activation."""
    acts = [np.asarray(X, np.float64)]
    for li, (W, b) in enumerate(params):
        z = acts[-1] @ W.T + b
        acts.append(z if li == len(params) - 1 else act(z))
    return acts


def query_with(cls_params, reg_params, rays, rho, wmax, t_mean, t_std, act, lam_lo=380.0,
               lam_hi=780.0, use_classifier=True):
    """query() with a given activation (the inference-time rational tanh)."""
    X, phi, mirror = features(rays.arrays() if hasattr(rays, "arrays") else rays, rho, wmax,
                              lam_lo, lam_hi)
    logit = forward_with(cls_params, X, act)[-1][:, 0]
    valid = (logit > 0.0) if use_classifier else np.ones(len(logit), bool)
    z = forward_with(reg_params, X, act)[-1]
    red = t_mean + t_std * z
    d = red[:, 2:5]
    red[:, 2:5] = d / np.linalg.norm(d, axis=1, keepdims=True)
    out = unreduce_outputs(red, phi, mirror)
    out[~valid] = 0.0
    return out, valid, logit
