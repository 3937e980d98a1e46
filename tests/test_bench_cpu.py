"""The bench's roofline arithmetic (host logic, no GPU): the per-half-sweep roof of the
contraction for each epilogue form, its sum over timed steps, the last CTA's tile share, and
the fraction the JSON line reports."""
import math

import pytest

import bench
import workloads

PK = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}


def test_epilogue_operation_counts():
    # direct: u*u - 1, times (u c), into the row sum; cube: v*v, times v into the row sum
    assert bench.epilogue_ops(False) == 3.0
    assert bench.epilogue_ops(True) == 2.0


def test_alu_peak_from_unit_counts():
    assert math.isclose(bench.alu_peak_tops(PK), 152 * 128 * 2000e6 / 1e12)


@pytest.mark.parametrize("cube", [False, True])
@pytest.mark.parametrize("prec,products", [("mixed", 3), ("bf16", 1), ("split3", 6)])
def test_half_sweep_roof_terms(cube, prec, products):
    w = workloads.preset("c3")
    N = float(w.grid_points)
    Mk = 16
    r = bench.half_sweep_roof_s(w, prec, Mk, PK, cube)
    assert math.isclose(r["tensor"], 2.0 * products * Mk * N / (PK["bf16_tflops"] * 1e12))
    assert math.isclose(r["alu"], (2.0 if cube else 3.0) * N / (bench.alu_peak_tops(PK) * 1e12))
    assert math.isclose(r["hbm"], 2.0 * products * Mk * sum(w.n) / (PK["hbm_gbs"] * 1e9))


def test_fp64_roof_terms():
    w = workloads.preset("c1")
    N = float(w.grid_points)
    r = bench.half_sweep_roof_s(w, "fp64", 12, PK)
    assert set(r) == {"fp64", "hbm"}
    assert math.isclose(r["hbm"], 8.0 * N / (PK["hbm_gbs"] * 1e9))


def test_step_roofline_sums_half_sweeps_per_form():
    # two steps: one direct, one cube; the fraction is the summed roof over the measured time
    w = workloads.preset("c3")
    stats = [dict(als_sweeps=10, cube_form=False), dict(als_sweeps=20, cube_form=True)]
    ranks = [16, 16]
    times_ms = [50.0, 70.0]
    out = bench.step_roofline(w, "mixed", ranks, stats, times_ms, PK, "test", None)
    roof = {}
    for mk, st in zip(ranks, stats):
        for k, v in bench.half_sweep_roof_s(w, "mixed", mk, PK, st["cube_form"]).items():
            roof[k] = roof.get(k, 0.0) + st["als_sweeps"] * w.dim * v
    t = sum(times_ms) / 1e3
    bound = max(roof, key=roof.get)
    assert out["bound"] == bound
    assert math.isclose(out["frac"], roof[bound] / t)
    if bound == "alu":
        ops = (3.0 * 10 + 2.0 * 20) * w.dim * w.grid_points
        assert math.isclose(out["achieved"], ops / t / 1e12)


def test_last_cta_tile_share_matches_the_split():
    # the first 16 CTAs weigh 1, the others 8; CTA c starts at floor(T cum(c) / cum(G))
    w = workloads.preset("c3")
    T = 1
    for d in range(w.dim):
        T *= -(-w.n[d] // 128)
    cum = lambda c: c if c <= 16 else 16 + 8 * (c - 16)
    lo = T * cum(151) // cum(152)
    assert math.isclose(bench.last_cta_tile_share(w), (T - lo) / T)
    # heavy CTAs hold eight times a light CTA's share: about 8 / (16 + 8 * 136) of the tiles
    assert abs(bench.last_cta_tile_share(w) - 8.0 / (16 + 8 * 136)) < 1e-3


@pytest.mark.parametrize("cube", [False, True])
def test_contraction_roof_of_the_last_cta(cube):
    w = workloads.preset("c3")
    r = bench.contraction_roof_us(w, 16.0, PK, "mixed", cube)
    n_cta = w.grid_points * bench.last_cta_tile_share(w)
    assert math.isclose(r["alu_us"], 1e6 * (2.0 if cube else 3.0) * n_cta / (128 * 2000e6))
    assert math.isclose(r["tensor_us"], 1e6 * 2.0 * 3 * 16 * n_cta / (PK["bf16_tflops"] * 1e12 / 152))
    assert math.isclose(r["roof_us"], max(r["alu_us"], r["tensor_us"]))
