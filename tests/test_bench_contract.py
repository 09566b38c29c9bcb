"""The reference arm of bench.py on CPU: one JSON line with the contract's
keys, the oracle's figures as its value, and its e2e object; other ranks
print nothing.  The timed oracle sample is replaced by a stub so the test
takes milliseconds (the sample itself is the oracle, tested elsewhere)."""
import argparse
import json

import pytest


@pytest.fixture
def bench_mod(monkeypatch):
    import bench
    calls = []

    def fake_baseline(seconds_hint=20.0):
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


def test_reference_other_ranks_print_nothing(bench_mod, capsys, monkeypatch):
    bench, calls = bench_mod
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(_args(2, 1, gpus=2)) == 0
    assert capsys.readouterr().out.strip() == ""
    assert calls == []
