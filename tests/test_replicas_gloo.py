"""The N > 1 path of bench.py on CPU: replicas on world_size 2 gloo ranks (no GPU). Each rank runs
its own independent copy of the workload (the path needs no exchange between GPUs), so the only
cross-rank step is the timing aggregate: the slowest rank's time and the units of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (100 + 50 r) ms for 4800 (r + 1) points
    ms, units, value = bench.job_throughput(100.0 + 50.0 * rank, 4800.0 * (rank + 1), dist, "cpu")
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{ms} {units} {value}\n")
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, units, value = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert ms == 150.0  # max over ranks
        assert units == 4800.0 * 3  # units of all ranks
        assert value == pytest.approx(units / 0.150)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(200.0, 4800, None) == (200.0, 4800.0, 24000.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    args = bench.parse()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
