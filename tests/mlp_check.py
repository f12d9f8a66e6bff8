"""Ray-by-ray comparison of a learned-map query with the oracle's FP64
forward of the same parameters (oracle/mlp.py, Eq. 11 with the networks of
Sec. 4.2).

FP32 queries evaluate the same rational tanh as the oracle's reference
forward; what remains is FP32 rounding of seven 32-term dot products, a few
1e-6 relative in standardised units, so outputs are held to 3e-5 x each
output's standard deviation plus two FP32 ulps of the output, and the
classifier's decision is compared where |logit| > 1e-3.

BF16 / FP16 tensor-core queries are held, ray by ray and output by output,
to twice a first-order bound of the half-precision rounding, computed in
FP64 per ray from the oracle's activations (`half_bound`), u the unit
roundoff (2^-9 BF16, 2^-11 FP16):
  - local error of layer l's pre-activation: its input and its weights are
    rounded to the half type, the products accumulate in FP32 with the FP32
    bias: |dz_l| <= (2 u + 2^-19) |W_l| |a_{l-1}|;
  - local error of a hidden activation: z is rounded to the half type, and
    tanh.approx of the packed pair returns a half value within 3 u |a| of
    tanh (one rounding of the result plus the approximation):
    |da_l| <= (1 - a_l^2)(|dz_l| + u |z_l|) + 3 u |a_l|;
  - each local error reaches the output through the exact Jacobian of the
    rest of the network, G_l = d out / d a_l (back-propagated per ray), so
    to first order |d out| <= sum_l |G_l| |da_l| + |dz_L|;
  - outputs are de-standardised by the training set's standard deviations,
    positions rotated back to the ray's frame (a component's error at most
    the sum of both reduced components'), the direction renormalised (to
    first order a component's error at most the norm of the raw direction's
    error, itself at most the sum of its components', for a raw direction of
    unit length).
The classifier's decision is compared where the logit exceeds twice its own
bound; on rays both sides call valid, a position may miss by twice its
bound plus 1e-5 mm, a direction component by twice its bound plus 1e-6, I by
twice its bound plus 1e-6.  On random networks with this rounding simulated
in numpy the worst error is about a tenth of the bound, and a dropped bias
or a transposed layer exceeds twice the bound on most rays
(tests/test_mlp_bound.py)."""
import numpy as np

from oracle import mlp

U_HALF = {1: 2.0 ** -9, 2: 2.0 ** -11}      # LT_MLP_BF16, LT_MLP_F16


def half_bound(params, X, u):
    """(output [n, k], first-order error bound [n, k]) of the network
    [(W, b), ...] on X under half-precision rounding with unit roundoff u."""
    acts, zs = [np.asarray(X, np.float64)], []
    L = len(params)
    for li, (W, b) in enumerate(params):
        z = acts[-1] @ W.T + b
        zs.append(z)
        if li < L - 1:
            acts.append(np.tanh(z))
    local = []
    for li, (W, b) in enumerate(params):
        dz = (2.0 * u + 2.0 ** -19) * (np.abs(acts[li]) @ np.abs(W).T)
        if li == L - 1:
            local.append(dz)
        else:
            a = acts[li + 1]
            local.append((1.0 - a * a) * (dz + u * np.abs(zs[li])) + 3.0 * u * np.abs(a))
    bound = local[-1].copy()
    G = np.broadcast_to(params[-1][0], (len(acts[0]),) + params[-1][0].shape)   # d out / d a_{L-1}
    for li in range(L - 2, -1, -1):
        bound += np.einsum("nkj,nj->nk", np.abs(G), local[li])
        if li > 0:
            G = np.einsum("nkj,jm->nkm", G * (1.0 - acts[li + 1] ** 2)[:, None, :], params[li][0])
    return zs[-1], bound


def check_query(out, flags, reg, cls, rays, rho, wmax, t_mean, t_std, precision, label=""):
    """Assert the GPU's query (out [n, 6], flags [n]) of the networks (FP64
    [(W, b), ...]) on `rays` against the oracle; returns a report dict."""
    t_mean, t_std = np.asarray(t_mean, np.float64), np.asarray(t_std, np.float64)
    gv = (flags & 1) != 0
    if precision in (0, 3):
        oo, ov, logit = mlp.query_with(cls, reg, rays, rho, wmax, t_mean, t_std, mlp.tanh_lambert,
                                       use_classifier=precision == 0)
        clear = np.abs(logit) > 1e-3 if precision == 0 else np.ones(len(gv), bool)
        assert np.array_equal(gv[clear], ov[clear]), label
        both = gv & ov
        err = np.abs(out[both].astype(np.float64) - oo[both])
        tol = 3e-5 * t_std + 2 * 2.0 ** -23 * np.abs(oo[both])
        bad = [q for q in (0, 1, 5) if not np.all(err[:, q] <= tol[:, q])]
        assert not bad, (label, bad, err.max(axis=0))
        assert err.shape[0] == 0 or err[:, 2:5].max() < 3e-5, label
        rep = {"decided": float(clear.mean()), "compared": int(both.sum()),
               "err_max": err.max(axis=0).tolist() if len(err) else None}
    else:
        u = U_HALF[precision]
        oo, ov, logit = mlp.query(cls, reg, rays, rho, wmax, t_mean, t_std)
        X, _, _ = mlp.features(rays.arrays(), rho, wmax)
        _, elog = half_bound(cls, X, u)
        clear = np.abs(logit) > 2.0 * elog[:, 0]
        assert np.array_equal(gv[clear], ov[clear]), label
        _, ez = half_bound(reg, X, u)
        ez = ez * t_std
        bpos = 2.0 * (ez[:, 0] + ez[:, 1])
        bdir = 2.0 * ez[:, 2:5].sum(axis=1)
        bI = 2.0 * ez[:, 5]
        both = gv & ov
        err = np.abs(out.astype(np.float64) - oo)
        epos, edir = err[:, 0:2].max(axis=1), err[:, 2:5].max(axis=1)
        ok = (epos <= bpos + 1e-5) & (edir <= bdir + 1e-6) & (err[:, 5] <= bI + 1e-6)
        viol = both & ~ok
        rep = {"decided": float(clear.mean()), "compared": int(both.sum()), "violations": int(viol.sum())}
        if both.any():
            rep.update(pos_err_over_bound=float((epos[both] / bpos[both]).max()),
                       dir_err_over_bound=float((edir[both] / bdir[both]).max()),
                       I_err_over_bound=float((err[both, 5] / bI[both]).max()),
                       pos_bound_median_mm=float(np.median(bpos[both])))
        assert not viol.any(), (label, rep, np.nonzero(viol)[0][:5])
    assert np.all(out[~gv] == 0), label
    return rep
