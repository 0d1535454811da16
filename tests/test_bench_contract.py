"""bench.py's reference arm on the CPU: the FP64 oracle timed on a bounded sample of the tiny
workload prints one JSON line with the contract's keys (no GPU needed)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "0"])
    assert bench.main() == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_oracle_sample_extrapolates_from_measured_builds():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2412_17132_gb300 import synth

    r = bench.oracle_sample(synth.tiny(), n_points=1)
    assert r["t_full_s"] >= r["t_table_s"] > 0 and r["t_build_s"] > 0
    assert r["value"] == (1 * 400) / r["t_full_s"]  # one core, 400 grid points per step
