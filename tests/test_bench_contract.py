"""The reference arm of bench.py on CPU: one JSON line with the contract's
keys, the oracle's figures as its value, and its e2e object; other ranks
print nothing.  The timed oracle sample is replaced by a stub so the test
takes milliseconds (the sample itself is the oracle, tested elsewhere).
Also the roofline arithmetic of the GPU line: each workload's fine launch
in the unit its roof is stated in, the measured traffic scaled by slices."""
import argparse
import json

import pytest


@pytest.fixture
def bench_mod(monkeypatch):
    import bench
    calls = []

    def fake_baseline(name=None):
        calls.append(1)
        return {"value": 1.0e8 + len(calls), "unit": bench.UNIT, "cores": 4, "kind": "oracle",
                "sample": "stub sample"}

    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)
    return bench, calls


def _args(steps, warmup, gpus=1):
    return argparse.Namespace(steps=steps, warmup=warmup, gpus=gpus, impl="reference")


def test_reference_line(bench_mod, capsys, monkeypatch):
    bench, calls = bench_mod
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.run_reference(_args(3, 2)) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 5                       # warm-up and timed samples
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT
    assert line["value"] == pytest.approx(1.0e8 + 4)      # median of the 3 timed samples
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 4
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT,
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    # the headline workload, with the same config object as the GPU arm's
    assert line["config"]["grid"] == "40x40x40x2" and line["config"]["N"] == 256
    assert line["config"]["nF"] == 1000 and line["config"]["batch"] == 8
    assert "bruss3d" in line["config"]["workload"]
    assert line["config"]["precision"] == "mixed_bf16"
    assert line["config"] == bench.line_config("bruss3d", "mixed_bf16", 1)


def test_reference_line_names_its_workload(bench_mod, capsys, monkeypatch):
    bench, calls = bench_mod
    monkeypatch.delenv("RANK", raising=False)
    args = _args(1, 0)
    args.workload = "swe_box"
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["config"]["grid"] == "100x50x3" and line["config"]["N"] == 235
    assert line["config"]["nF"] == 35 and "walls" in line["config"]["workload"]
    assert line["config"] == bench.line_config("swe_box", "mixed", 1)
    assert bench.timed_precision("diffreact2d", None) == "mixed"


def test_cpu_sample_keeps_the_slice_length():
    """The oracle's bounded sample: the workload's grid, operator and slice
    length, one member, at most 16 slices and 2e9 cell-updates per
    iteration."""
    import bench
    import workloads as W
    for name in ("bruss3d", "diffreact2d", "bruss2d", "swe_box"):
        full = bench.bench_config(name)
        cfg, what = bench.cpu_sample_config(name)
        assert (cfg["nx"], cfg["ny"], cfg["nz"], cfg["param"]) == \
            (full["nx"], full["ny"], full["nz"], full["param"])
        assert cfg["batch"] == 1 and cfg["N"] == min(16, full["N"])
        dT = (full["tN"] - full["t0"]) / full["N"]
        assert abs((cfg["tN"] - cfg["t0"]) / cfg["N"] - dT) < 1e-12 * dT
        assert cfg["nG"] == full["nG"] and cfg["nF"] <= full["nF"]
        assert cfg["N"] * W.dim(cfg) * cfg["nF"] <= max(2e9, cfg["N"] * W.dim(cfg) * 50)
        assert name in what


def test_reference_other_ranks_print_nothing(bench_mod, capsys, monkeypatch):
    bench, calls = bench_mod
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(_args(2, 1, gpus=2)) == 0
    assert capsys.readouterr().out.strip() == ""
    assert calls == []


def test_dam_break_workload_recipe():
    """The paper's dam break as DESIGN states it: 10 x 5 box, 100 x 50
    cells, walls, N = 235 on [0, 20], G = Euler x 7, F steps by the CFL
    rule, m = 3; depth 1 plus the bivariate normal density of the column
    (mean (2.5, 1.5) in box coordinates, covariance 0.25 I), no momentum."""
    import math

    import numpy as np

    import bench
    import workloads as W
    cfg = W.config("swe_box")
    assert (cfg["nx"], cfg["ny"], cfg["lx"], cfg["ly"]) == (100, 50, 10.0, 5.0)
    assert (cfg["N"], cfg["tN"], cfg["nG"], cfg["m"], cfg["bc"]) == (235, 20.0, 7, 3, "neumann")
    assert cfg["nF"] == W.swe_steps(cfg)[0] == 35
    u0 = W.initial_condition(cfg)[0]
    n = 100 * 50
    h = u0[:n].reshape(50, 100)
    assert np.all(u0[n:] == 0.0)
    j, i = np.unravel_index(np.argmax(h), h.shape)
    assert abs((i + 0.5) * 0.1 - 2.5) <= 0.05 and abs((j + 0.5) * 0.1 - 1.5) <= 0.05
    assert h.max() <= 1.0 + 1.0 / (2 * math.pi * 0.25) + 1e-12
    assert h.min() >= 1.0
    # the column's volume above depth 1 is the density's mass inside the
    # box: the bottom wall is 3 sigma below the centre, the others farther
    phi = lambda z: 0.5 * math.erfc(-z / math.sqrt(2.0))
    inside = (phi(15.0) - phi(-5.0)) * (phi(7.0) - phi(-3.0))
    assert abs((h - 1.0).sum() * 0.1 * 0.1 - inside) < 1e-4   # midpoint rule, h = 0.1
    assert "walls" in bench.describe(cfg) and "F=RK4x35" in bench.describe(cfg)


PK = {"hbm_gbs": 6662.6, "sm_max_mhz": 2070.0}
WIDE = {"cluster": 10, "threads": 800, "px": 2, "rs": 4}


def test_roofline_of_the_headline_in_bytes_per_cell_step():
    """The 3D Brusselator's fine launch against HBM in the workload's unit,
    8 B per cell-step, and against the FP32 ALU with every operation counted."""
    import bench
    cells, launch_s, slices = 2.518e11, 1.3407, 1967.0
    r = bench.roofline("bruss3d", cells, launch_s, WIDE, slices, PK)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and "_wide" in r["kernel"]
    assert r["achieved"] == pytest.approx(cells * 8 / launch_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6662.6)
    assert r["traffic"] == pytest.approx(16448512 / 16 * slices)
    alu = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["alu_recount"]["flop_per_cell_step"] == (4 * (21 + 18) + 2 * 13) / 2.0
    assert r["alu_recount"]["frac"] == pytest.approx(cells * 91 / launch_s / 1e12 / alu)


def test_roofline_of_the_other_workloads_in_their_units():
    """Diffusion-reaction against the FP32 ALU at 40 flop per cell-step,
    Burgers (all FP64) against the nominal FP64 rate at 60 flop."""
    import bench
    tf = {"cluster": 16, "threads": 128, "px": 2, "rs": 4}
    r = bench.roofline("diffreact2d", 1e11, 0.5, tf, 64, PK)
    alu = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(1e11 * 40 / 0.5 / 1e12 / alu)
    assert r["traffic"] == pytest.approx(16838144.0)
    fp64 = {"cluster": 1, "threads": 64, "px": 0, "rs": 0, "R": 2}
    r = bench.roofline("burgers1d", 1e9, 0.5, fp64, 16, PK)
    assert r["bound"] == "alu" and r["peak"] == 1.25
    assert r["frac"] == pytest.approx(1e9 * 60 / 0.5 / 1e12 / 1.25)
    assert "alu_recount" not in r and r["traffic"] is None
    # a tiling without a capture reports no traffic
    r = bench.roofline("bruss3d", 1e11, 1.0, dict(WIDE, cluster=8, rs=5), 100, PK)
    assert r["traffic"] is None
