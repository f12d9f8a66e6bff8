"""CPU checks of the benchmark's own arithmetic: the roofline objects it
reports (algorithmic bytes or counted flop over a kernel's measured time),
the derived FP32 peak, the map-error statistics and the oracle baseline's
split of a batch over host threads."""
import math

import numpy as np
import pytest

import bench
import oracle
from paper_2605_04017_gb300 import workloads as w

PEAKS = {"hbm_gbs": 6784.8, "src": "measured", "sm_max_mhz": 2070.0}


def test_fp32_peak_is_the_unit_count_times_the_clock():
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_hbm_roofline_divides_algorithmic_bytes_by_kernel_time():
    # 20 steps, one launch each, 0.1443 ms per launch; 399,961,823 bytes per step
    prof = {"map_query_kernel": (20, 20 * 0.1443, 0)}
    r = bench.kernel_roofline("map_query_kernel", prof, PEAKS, 20, units_bytes=399961823)
    achieved = 399961823 / 0.1443e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(achieved, abs=0.1)
    assert r["frac"] == pytest.approx(achieved / 6784.8, abs=1e-4)
    assert r["launches_per_step"] == 1.0 and r["kernel_ms_per_step"] == pytest.approx(0.1443)


def test_alu_roofline_counts_flop_per_interaction():
    # 2 launches per step (a wave split in two), 19,099,764 interactions per step
    prof = {"trace_kernel": (40, 20 * 0.1811, 20 * 19099764)}
    r = bench.kernel_roofline("trace_kernel", prof, PEAKS, 20, flops_per_work=89)
    achieved = 19099764 * 89 / 0.1811e-3 / 1e12
    assert r["bound"] == "alu" and r["launches_per_step"] == 2.0
    assert r["achieved"] == pytest.approx(achieved, abs=0.01)
    assert r["frac"] == pytest.approx(achieved / bench.fp32_peak_tflops(2070.0), abs=1e-4)
    assert r["interactions_per_step"] == 19099764


def test_pos_err_uses_rays_valid_on_both_sides_and_skips_grazing():
    a = np.zeros((5, 6), np.float32)
    b = np.zeros((5, 6), np.float32)
    a[:, 0] = [0.0, 3.0, 1.0, 0.0, 0.0]
    a[:, 1] = [0.0, 4.0, 0.0, 0.0, 9.0]
    af = np.array([1, 1, 1, 0, 1], np.uint8)
    bf = np.array([1, 1, 1, 1, 1 | 0x40], np.uint8)     # ray 4 is grazing on the reference side
    e = bench.pos_err(a, af, b, bf, 1)
    d = np.array([0.0, 5.0, 1.0])
    assert e["rms_mm"] == pytest.approx(math.sqrt((d ** 2).mean()))
    assert e["p99_mm"] == pytest.approx(np.percentile(d, 99))
    assert e["valid_agreement"] == pytest.approx(4 / 5)


def test_oracle_threads_split_covers_the_batch():
    # the batch goes to k threads in k contiguous parts that tile it exactly,
    # each with its rays' classes, and the parts' answers equal one call's
    from oracle import poly
    p = w.singlet_lens()
    om = poly.PolyMap(p, (0, 0), 12.0, bench.SMAX, 380.0, 780.0, 3, (2, 2, 1, 1), (2, 2, 2, 1), 5, tol=1e-4)
    rays = w.singlet_rays(1001)
    inside, cells = om.locate(rays)
    classes = np.full(len(rays), 2, np.uint8)
    classes[inside] = om.cell_class[tuple(cells[inside].T)]
    whole, wf = om.query(rays, classes=classes)
    parts = []

    class Spy:
        def query(self, r, classes=None):
            parts.append((r.arrays()[0].copy(), classes.copy(), om.query(r, classes=classes)))

    dt = bench.oracle_query_threads(Spy(), rays, classes, 3)
    assert dt > 0 and len(parts) == 3
    x = rays.arrays()[0]
    start = {int(np.flatnonzero(x == px[0])[0]): (px, c, res) for px, c, res in parts}
    assert sorted(len(px) for px, _, _ in parts) == [333, 334, 334]
    pos = 0
    for s0 in sorted(start):
        px, c, (o, f) = start[s0]
        assert s0 == pos and np.array_equal(px, x[pos:pos + len(px)])
        assert np.array_equal(c, classes[pos:pos + len(px)])
        assert np.array_equal(o, whole[pos:pos + len(px)]) and np.array_equal(f, wf[pos:pos + len(px)])
        pos += len(px)
    assert pos == len(rays)


def test_map_error_statistics():
    class F:
        FLAG_VALID, FLAG_TRACED, FLAG_NEAR_EDGE = 1, 0x10, 2
    q = np.zeros((5, 6), np.float32)
    t = np.zeros((5, 6), np.float32)
    q[0, :2] = [3e-5, -4e-5]
    q[1, 2] = 2e-7
    q[2, 5] = 1e-6
    qf = np.array([1, 1, 1, 1 | 0x10, 0], np.uint8)    # ray 3 traced, ray 4 INVALID
    tf = np.array([1, 1, 1, 1, 1 | 2], np.uint8)        # ray 4 valid, near an edge
    e = bench.map_error(q, qf, t, tf, F)
    assert e["rays_interpolated"] == 3 and e["validity_mismatches"] == 1
    assert e["validity_mismatches_near_edge"] == 1
    assert e["pos_max_mm"] == pytest.approx(4e-5) and e["pos_euclid_max_mm"] == pytest.approx(5e-5, rel=1e-6)
    assert e["dir_max"] == pytest.approx(2e-7) and e["I_max"] == pytest.approx(1e-6)
