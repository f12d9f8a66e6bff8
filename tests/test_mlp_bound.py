"""CPU check of the half-precision error bound that the learned-map parity
tests hold the tensor-core queries to (tests/mlp_check.py): a forward pass
that rounds exactly where the bound assumes (inputs and weights to BF16 or
FP16, FP32 accumulation with FP32 biases, z rounded before tanh, the
activation rounded after it) stays within half the bound on random networks, both
Xavier-initialised and with weights scaled up until most hidden units
saturate; and a forward pass with a planted mistake (a dropped bias, a transposed
layer) exceeds twice the bound on most rays."""
import numpy as np
import pytest

from oracle import mlp

from mlp_check import U_HALF, half_bound


def to_bf16(x):
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def to_f16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)


def rounded_forward(params, X, rnd):
    a = rnd(X)
    for li, (W, b) in enumerate(params):
        z = (a.astype(np.float32) @ rnd(W).T.astype(np.float32)).astype(np.float64) + np.float32(b)
        z = z.astype(np.float32).astype(np.float64)
        if li == len(params) - 1:
            return z
        a = rnd(np.tanh(rnd(z)))
    raise ValueError


@pytest.mark.parametrize("precision,rnd", [(1, to_bf16), (2, to_f16)])
@pytest.mark.parametrize("scale", [1.0, 3.0])
@pytest.mark.parametrize("kind", ["reg", "cls"])
def test_rounded_forward_within_half_bound(precision, rnd, scale, kind):
    rng = np.random.Generator(np.random.PCG64(17))
    params = [(W * scale, rng.uniform(-0.3, 0.3, size=b.shape)) for W, b in mlp.init_params(kind, rng)]
    X = rng.uniform(-1.0, 1.0, size=(4000, 4))
    exact = mlp.forward(params, X)[-1]
    got = rounded_forward(params, X, rnd)
    _, bound = half_bound(params, X, U_HALF[precision])
    ratio = np.abs(got - exact) / bound
    print(kind, precision, scale, "max error / bound", ratio.max())
    assert ratio.max() <= 0.5


def planted(params, what):
    bad = [(W.copy(), b.copy()) for W, b in params]
    if what == "dropped bias":
        bad[3] = (bad[3][0], np.zeros_like(bad[3][1]))
    elif what == "transposed layer":
        bad[2] = (bad[2][0].T.copy(), bad[2][1])
    return bad


@pytest.mark.parametrize("what", ["dropped bias", "transposed layer"])
def test_planted_mistake_exceeds_half_bound(what):
    rng = np.random.Generator(np.random.PCG64(18))
    params = [(W, rng.uniform(-0.3, 0.3, size=b.shape)) for W, b in mlp.init_params("reg", rng)]
    X = rng.uniform(-1.0, 1.0, size=(4000, 4))
    exact = mlp.forward(params, X)[-1]
    got = rounded_forward(planted(params, what), X, to_bf16)
    _, bound = half_bound(params, X, U_HALF[1])
    assert (np.abs(got - exact) > 2.0 * bound).any(axis=1).mean() > 0.5
