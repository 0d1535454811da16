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


def test_chi0_executed_work_ratio_counts_the_launched_tiles(monkeypatch):
    """bench.py's executed-to-algorithmic MMA work of the chi0 kernels equals a brute-force count over the
    tiles the kernels launch (pair kernel: 256-row blocks p holding 128-column blocks 0 .. 2p + 1, the last
    up to the padded width; one-CTA kernel: the 128 x 128 blocks of the padded lower triangle), and those
    tiles cover every element of the lower triangle exactly once."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    n_ov = 640  # a multiple of the 64-wide K chunk: no K padding
    for n_aux in (1, 70, 128, 129, 300, 520, 700, 1100):
        pad = -(-n_aux // 128) * 128
        nqb, npb = pad // 128, -(-pad // 256)
        pair = [(256 * p, 128 * q, 256) for p in range(npb) for q in range(min(2 * p + 2, nqb))]
        single = [(128 * a, 128 * b, 128) for a in range(nqb) for b in range(a + 1)]
        for kernel, tiles in (("pair", pair), ("single", single)):
            cover = np.zeros((n_aux, n_aux), dtype=np.int32)
            for r0, c0, h in tiles:
                i = np.arange(r0, min(r0 + h, n_aux))[:, None]
                j = np.arange(c0, min(c0 + 128, n_aux))[None, :]
                cover[i, j] += 1
            low = np.tril(np.ones((n_aux, n_aux), dtype=bool))
            assert np.all(cover[low] == 1), (kernel, n_aux)  # each lower element by exactly one tile
            executed = sum(h * 128 for _, _, h in tiles) * n_ov
            if kernel == "single":
                monkeypatch.setenv("GWC_CHI0_KERNEL", "single")
            else:
                monkeypatch.delenv("GWC_CHI0_KERNEL", raising=False)
            name, ratio = bench.chi0_kernel_info(n_aux, n_ov)
            assert name == ("chi0_pair_kernel" if kernel == "pair" else "chi0_tc_kernel")
            # algorithmic: N_aux (N_aux + 1) / 2 elements x N_ov products
            assert abs(ratio - executed / (n_aux * (n_aux + 1) / 2 * n_ov)) < 1e-12
