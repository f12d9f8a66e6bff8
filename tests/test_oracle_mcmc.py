"""Pins of the oracle's valid-region sampler (Sec. 5.1, data collection):
SplitMix64 against its reference outputs, the chains' stationary law
against rejection sampling of the same target, and chain invariants."""
import math

import numpy as np
import pytest

import oracle
from oracle import mcmc
from paper_2605_04017_gb300 import workloads as w

SM = math.tan(math.radians(10.0))
LO, HI = [-12.0, -12.0, -SM, -SM, 380.0], [12.0, 12.0, SM, SM, 780.0]


def test_splitmix64_reference_outputs():
    # the generator's first three outputs from state 0 (state advanced by gamma per call)
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [int(mcmc.splitmix64(np.uint64((k * g) % (1 << 64)))) for k in range(3)]
    assert got == want


def test_uniforms_are_24_bit_and_in_range():
    u = mcmc.uniforms(7, np.arange(100000), 3, 2)
    assert u.dtype == np.float32 and (u >= 0).all() and (u < 1).all()
    assert np.all(u * 2 ** 24 == np.round(u * 2 ** 24))
    assert abs(u.mean() - 0.5) < 0.005


def run(path=(0, 0), chains=3000, steps=60, small=0.05, p_large=0.1, seed=5):
    ol = oracle.Lens(w.singlet_lens())
    return ol, mcmc.sample(ol, path, LO, HI, seed, chains, steps, small, p_large, 64, w.Rays)


@pytest.mark.parametrize("path", [(0, 0), (1, 2)])
def test_stationary_law_is_uniform_over_the_valid_region(path):
    """Marginals of the chains (after burn-in) against rejection sampling of
    the same binary target (two-sample KS test)."""
    stats = pytest.importorskip("scipy.stats")
    ol, (u, started, acc, _) = run(path, chains=6000)
    assert started.mean() > 0.99
    # chains start on the target (their first state is a valid uniform draw)
    # and are independent of one another: the chains' states at one step are
    # independent draws from the stationary law, whatever the correlation
    # along a chain
    samp = u[-1, started]
    rng = np.random.default_rng(11)
    cand = np.stack([rng.uniform(LO[d], HI[d], 400000) for d in range(5)], 1).astype(np.float32)
    _, v, _, _ = ol.trace(w.Rays(*mcmc.state_rays(cand)), path)
    ref = cand[v == 1]
    assert len(ref) > 10000
    for d in range(5):
        p = stats.ks_2samp(samp[:, d], ref[:, d]).pvalue
        assert p > 1e-4, (path, d, p)


def test_chain_invariants():
    ol, (u, started, acc, _) = run(chains=500, steps=30)
    s = u[:, started].reshape(-1, 5)
    assert (s >= np.float32(LO)).all() and (s <= np.float32(HI)).all()
    _, v, _, _ = ol.trace(w.Rays(*mcmc.state_rays(s)), (0, 0))
    assert (v == 1).all()                                  # a chain only visits valid rays
    assert (acc[started] <= 30).all() and acc[started].mean() > 5


def test_independent_proposals_keep_exactly_the_valid_draws():
    """With p_large = 1 every proposal is the independent uniform draw of the
    step, so a chain moves to it iff that draw's ray is valid."""
    ol, (u, started, acc, _) = run(chains=400, steps=5, p_large=1.0)
    lo_f, hi_f, w_f = mcmc.box_f32(LO, HI)
    C = np.arange(400)
    prev = None
    for s in range(5):
        i = 64 + s
        draw = np.stack([lo_f[d] + mcmc.uniforms(5, C, i, 1 + d) * w_f[d] for d in range(5)], 1)
        _, v, _, _ = ol.trace(w.Rays(*mcmc.state_rays(draw)), (0, 0))
        moved = started & (v == 1)
        assert np.array_equal(u[s][moved], draw[moved])
        if prev is not None:
            stay = started & (v != 1)
            assert np.array_equal(u[s][stay], prev[stay])
        prev = u[s]


def test_zero_step_chains_do_not_move():
    ol, (u, started, acc, _) = run(chains=200, steps=4, small=0.0, p_large=0.0)
    assert np.array_equal(u[0][started], u[3][started])
    assert (acc[started] == 4).all()
