"""CPU checks of the parity checker itself (tests/parity.py), so that a GPU
parity test cannot pass vacuously: the oracle's own results, rounded to
FP32 as the kernels store them, pass; a planted error in any output, in the
validity mask of an unflagged ray, in an invalid ray's zeros or in the
bad-input flag fails; a mask difference on a ray flagged near an aperture
edge is accepted."""
import numpy as np
import pytest

import oracle
from paper_2605_04017_gb300 import workloads as w

from parity import DIR_TOL, F_EDGE, F_VALID, I_TOL, POS_TOL, compare_trace


@pytest.fixture(scope="module")
def traced():
    p = w.singlet_lens()
    ol = oracle.Lens(p)
    rays = w.singlet_rays(5000)
    ex, ev, edge, kmin = ol.trace(rays, (0, 0))
    out = np.where((ev == 1)[:, None], ex, 0.0).astype(np.float32)
    flags = np.where(ev == 1, F_VALID, np.where(ev == 8, 8, 0)).astype(np.uint8)
    return out, flags, ex, ev, edge, kmin


def pick(traced, valid=True):
    out, flags, ex, ev, edge, kmin = traced
    ok = (ev == 1) if valid else (ev == 0)
    ok &= (edge >= 1e-3) & (kmin >= 0.1)
    return int(np.flatnonzero(ok)[len(np.flatnonzero(ok)) // 2])


def test_oracle_results_in_fp32_pass(traced):
    out, flags, ex, ev, edge, kmin = traced
    st = compare_trace(out, flags, ex, ev, edge, kmin, "clean")
    assert st["valid_gpu"] > 1000 and st["mask_mismatch"] == 0


@pytest.mark.parametrize("col,delta", [(0, 2 * POS_TOL), (1, -2 * POS_TOL), (3, 2 * DIR_TOL),
                                       (4, -2 * DIR_TOL), (5, 2 * I_TOL)])
def test_a_planted_output_error_fails(traced, col, delta):
    out, flags, ex, ev, edge, kmin = traced
    bad = out.copy()
    r = pick(traced)
    bad[r, col] = np.float32(np.float64(bad[r, col]) + delta)
    with pytest.raises(AssertionError):
        compare_trace(bad, flags, ex, ev, edge, kmin, "planted")


def test_a_flipped_mask_bit_fails_unless_flagged(traced):
    out, flags, ex, ev, edge, kmin = traced
    r = pick(traced, valid=False)
    f = flags.copy()
    o = out.copy()
    f[r] |= F_VALID
    o[r] = ex[r] if np.any(ex[r]) else np.float32(1.0)
    with pytest.raises(AssertionError):
        compare_trace(o, f, ex, ev, edge, kmin, "flipped")
    # the same difference on a ray the GPU flags as near an edge is explained
    r2 = pick(traced, valid=True)
    f2 = flags.copy()
    o2 = out.copy()
    f2[r2] = F_EDGE          # reported invalid, flagged near an edge
    o2[r2] = 0.0
    st = compare_trace(o2, f2, ex, ev, edge, kmin, "flagged")
    assert st["mask_mismatch"] == 1 and st["mask_mismatch_unflagged"] == 0


def test_nonzero_outputs_of_an_invalid_ray_fail(traced):
    out, flags, ex, ev, edge, kmin = traced
    r = pick(traced, valid=False)
    o = out.copy()
    o[r, 5] = np.float32(0.5)
    with pytest.raises(AssertionError):
        compare_trace(o, flags, ex, ev, edge, kmin, "nonzero")


def test_a_bad_input_flag_mismatch_fails(traced):
    out, flags, ex, ev, edge, kmin = traced
    r = pick(traced, valid=False)
    f = flags.copy()
    f[r] |= 8
    with pytest.raises(AssertionError):
        compare_trace(out, f, ex, ev, edge, kmin, "bad-input")


@pytest.fixture(scope="module")
def ghost():
    """The singlet's ghost (1, 2): many of its valid rays leave near grazing."""
    p = w.singlet_lens()
    ol = oracle.Lens(p)
    rays = w.singlet_rays(20000)
    ex, ev, edge, kmin = ol.trace(rays, (1, 2))
    out = np.where((ev == 1)[:, None], ex, 0.0).astype(np.float32)
    flags = np.where(ev == 1, F_VALID, np.where(ev == 8, 8, 0)).astype(np.uint8)
    return ol, rays, out, flags, ex, ev, edge, kmin


def test_a_planted_error_on_a_grazing_ray_fails(ghost):
    """Grazing rays are held to a bound too: an error that neither the
    tolerance nor the oracle's own sensitivity explains fails."""
    ol, rays, out, flags, ex, ev, edge, kmin = ghost
    g = np.flatnonzero((ev == 1) & (kmin < 1e-2) & (edge > 1e-3))
    assert g.size > 0
    r = int(g[0])
    st = compare_trace(out, flags, ex, ev, edge, kmin, "clean ghost", cond=(ol, rays, (1, 2)))
    assert st["grazing"] > 0 and st["value_violations"] == 0
    for col, delta in ((0, 0.5), (2, 1e-2), (5, 1e-3)):
        bad = out.copy()
        bad[r, col] = np.float32(np.float64(bad[r, col]) + delta)
        with pytest.raises(AssertionError):
            compare_trace(bad, flags, ex, ev, edge, kmin, "planted grazing", cond=(ol, rays, (1, 2)))


def test_a_planted_error_on_a_flagged_valid_ray_fails(traced):
    """A near-edge flag exempts a ray's validity bit, never its values."""
    out, flags, ex, ev, edge, kmin = traced
    r = pick(traced)
    f = flags.copy()
    f[r] |= F_EDGE
    bad = out.copy()
    bad[r, 0] = np.float32(np.float64(bad[r, 0]) + 2 * POS_TOL)
    with pytest.raises(AssertionError):
        compare_trace(bad, f, ex, ev, edge, kmin, "planted flagged")
