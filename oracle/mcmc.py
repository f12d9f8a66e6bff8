"""ORACLE -- test infrastructure only (see oracle/__init__.py).

The valid-region sampler of Sec. 5.1 (data collection): for most paths only
a small fraction of the input space gives valid rays, so training rays are
drawn with a Markov chain Monte Carlo sampler whose target is the binary
visibility of the path -- 1 for an entrance ray that reaches the image
plane along the path, 0 otherwise.  Readings (the paper gives the target
and its citation only):
  - the state is a point u = (x, y, s_x, s_y, lambda) of the lattice box
    [lo, hi]; its entrance ray is (x, y) with direction
    normalize(s_x, s_y, 1) and wavelength lambda, all FP32, the direction
    rounded exactly as a lattice node's;
  - a step proposes, with probability p_large, an independent uniform
    point of the box, else a uniform point of the box of half-width
    small * (hi - lo) around u (both proposals are symmetric), and accepts
    it iff it lies in the box and its ray is valid -- the Metropolis rule
    for a binary target, so the chain's stationary law is uniform over the
    valid region;
  - a chain starts at the first valid independent uniform point of at most
    init_tries draws, or never starts;
  - random numbers: u(chain, i, k) = top 24 bits of SplitMix64(seed +
    (chain << 32 | i << 3 | k)) * 2^-24, with i the draw (init try t: i = t;
    chain step s: i = init_tries + s) and k the coordinate (0: the
    large/small choice, 1..5: the five dimensions).  SplitMix64 is Steele,
    Lea and Flood's (2014) generator: z += 0x9E3779B97F4A7C15, then two
    xor-shift-multiply rounds and a final xor-shift.
Proposals are computed in FP32 with one rounding per operation, so a GPU
implementation of the same reading reproduces the chains bit for bit
wherever the two tracers agree on validity.

Parity status: pinned (SplitMix64 reference outputs, uniform-law
agreement with rejection sampling on a lens whose valid region is known,
chain invariants).
"""
from __future__ import annotations

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def splitmix64(z):
    """SplitMix64 of a uint64 array (or int): the mix of z + gamma (arithmetic
    modulo 2^64)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(z, dtype=np.uint64) + np.uint64(_GAMMA))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, chains: np.ndarray, i: int, k: int) -> np.ndarray:
    """FP32 uniforms in [0, 1) for the given chains, draw i, coordinate k."""
    ctr = (chains.astype(np.uint64) << np.uint64(32)) | np.uint64((i << 3) | k)
    with np.errstate(over="ignore"):
        h = splitmix64((np.uint64(seed) + ctr) & np.uint64(_MASK))
    return ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def box_f32(lo, hi):
    lo_f = np.asarray(lo, np.float64).astype(np.float32)
    hi_f = np.asarray(hi, np.float64).astype(np.float32)
    w_f = (np.asarray(hi, np.float64) - np.asarray(lo, np.float64)).astype(np.float32)
    return lo_f, hi_f, w_f


def state_rays(u):
    """Entrance rays (x, y, dx, dy, dz, lambda) of states u[n, 5], FP32 with one
    rounding per operation: a = s_x^2, b = s_y^2, len = sqrt((a + b) + 1)."""
    u = np.asarray(u, np.float32)
    sx, sy = u[:, 2], u[:, 3]
    a = sx * sx
    b = sy * sy
    n2 = (a + b) + np.float32(1.0)
    ln = np.sqrt(n2)
    return [u[:, 0].copy(), u[:, 1].copy(), sx / ln, sy / ln, np.float32(1.0) / ln, u[:, 4].copy()]


def sample(lens, path, lo, hi, seed: int, chains: int, steps: int, small: float, p_large: float,
           init_tries: int, rays_type, edge_eps: float = 1e-6, tir_eps: float = 1e-6):
    """Run the chains.  Returns (u[steps, chains, 5] states after each step,
    started[chains] bool, accepted[chains] counts, first_amb[chains]): the
    last is the first draw (init try t: t; step s: init_tries + s) whose
    validity decision lay within edge_eps of an aperture edge or tir_eps of
    total internal reflection (a large number if none) -- the decisions an
    FP32 tracer may take differently.  `lens` is an oracle Lens; rays_type
    builds a Rays from six arrays."""
    lo_f, hi_f, w_f = box_f32(lo, hi)
    h_f = (np.float32(small) * w_f).astype(np.float32)
    C = np.arange(chains)
    u = np.zeros((chains, 5), np.float32)
    started = np.zeros(chains, bool)
    never = np.iinfo(np.int64).max
    first_amb = np.full(chains, never, np.int64)

    def valid(states, idx, chain_ids, draw):
        if len(idx) == 0:
            return np.zeros(0, bool)
        _, v, edge, kmin = lens.trace(rays_type(*state_rays(states[idx])), path)
        amb = (edge < edge_eps) | (np.abs(kmin) < tir_eps)
        c = chain_ids[idx][amb]
        first_amb[c] = np.minimum(first_amb[c], draw)
        return v == 1

    for t in range(init_tries):
        todo = np.nonzero(~started)[0]
        if len(todo) == 0:
            break
        cand = np.stack([lo_f[d] + uniforms(seed, C[todo], t, 1 + d) * w_f[d] for d in range(5)], 1)
        ok = valid(cand.astype(np.float32), np.arange(len(todo)), todo, t)
        u[todo[ok]] = cand[ok]
        started[todo[ok]] = True
    out = np.zeros((steps, chains, 5), np.float32)
    acc = np.zeros(chains, np.int64)
    run = np.nonzero(started)[0]
    for s in range(steps):
        i = init_tries + s
        large = uniforms(seed, C[run], i, 0) < np.float32(p_large)
        prop = np.empty((len(run), 5), np.float32)
        for d in range(5):
            xi = uniforms(seed, C[run], i, 1 + d)
            big = lo_f[d] + xi * w_f[d]
            near = u[run, d] + (np.float32(2.0) * xi - np.float32(1.0)) * h_f[d]
            prop[:, d] = np.where(large, big, near)
        inside = np.all((prop >= lo_f) & (prop <= hi_f), axis=1)
        ok = np.zeros(len(run), bool)
        ins = np.nonzero(inside)[0]
        ok[ins] = valid(prop, ins, run, i)
        u[run[ok]] = prop[ok]
        acc[run[ok]] += 1
        out[s] = u
    return out, started, acc, first_amb
