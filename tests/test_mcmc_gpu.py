"""lt_mcmc_sample (the valid-region sampler of Sec. 5.1) against the oracle's
chains, chain by chain and step by step.  Both sides draw the same
counter-based uniforms and compute proposals with the same FP32 operations,
so every state is bit-for-bit equal until a chain meets a proposal whose
validity lies within 1e-6 mm of an aperture edge or 1e-6 of total internal
reflection (where the FP32 and FP64 tracers may decide differently); such a
chain is compared up to that step only."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mcmc
from paper_2605_04017_gb300 import lt, workloads as w

pytestmark = pytest.mark.gpu

SM = math.tan(math.radians(10.0))


def oracle_accept(p):
    try:
        e, b = oracle.Lens(p).paraxial(w.LAMBDA_D_NM)
        return e > 0 and b > 0
    except ValueError:
        return False


def compare(presc, path_id, rho, chains, steps, small, p_large, init_tries, seed):
    lo, hi = [-rho, -rho, -SM, -SM, 380.0], [rho, rho, SM, SM, 780.0]
    lens = lt.Lens(presc)
    ol = oracle.Lens(presc)
    path = oracle.path_ij(presc.n_surfaces, path_id)
    f, flags, acc = lt.mcmc_sample(lens, path_id, lo, hi, seed, chains, steps, small, p_large, init_tries)
    torch.cuda.synchronize()
    g = np.stack([t.cpu().numpy()[: chains * steps].reshape(steps, chains) for t in f], -1)   # [steps, chains, 6]
    gfl = flags.cpu().numpy()[: chains * steps].reshape(steps, chains)
    gacc = acc.cpu().numpy()[:chains]
    u, started, oacc, first_amb = mcmc.sample(ol, path, lo, hi, seed, chains, steps, small, p_large, init_tries,
                                              w.Rays)
    clean_start = first_amb >= init_tries              # no ambiguous decision while starting
    assert np.array_equal(((gfl[0] & 1) != 0)[clean_start], started[clean_start])
    compared = 0
    for c in np.nonzero(started & clean_start)[0]:
        last = min(steps, int(first_amb[c]) - init_tries)   # steps decided before any ambiguity
        if last <= 0:
            continue
        ref = np.stack(mcmc.state_rays(u[:last, c]), -1)
        assert np.array_equal(g[:last, c], ref), f"chain {c} differs before step {last}"
        compared += last
        if last == steps:
            assert gacc[c] == oacc[c]
    n_amb = int((first_amb < init_tries + steps).sum())
    print(f"path {path_id}: {int(started.sum())} chains started of {chains}, {compared} states compared, "
          f"{n_amb} chains met an ambiguous decision, acceptance {oacc[started].mean() / steps:.3f}")
    assert compared > 0.9 * started.sum() * steps
    return started.mean()


def test_singlet_main_and_ghost_chains_match_oracle():
    p = w.singlet_lens()
    compare(p, 0, 12.0, 4096, 32, 0.05, 0.1, 32, 7)
    compare(p, 1, 12.0, 4096, 32, 0.05, 0.1, 32, 8)


def test_eleven_surface_ghost_chains_match_oracle():
    p = w.eleven_surface_lens(oracle_accept)
    rho = w.eleven_rho(p)
    # a ghost with a small valid fraction: chains find it where uniform draws rarely do
    frac = compare(p, 20, rho, 2048, 24, 0.03, 0.05, 64, 9)
    assert frac > 0.05
