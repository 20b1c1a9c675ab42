"""bench.py's multi-process logic on CPU: two gloo ranks agree on the slowest rank's time (max over ranks),
the whole-job rate counts every rank's units, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                   # rank 1 is the slowest
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.job_rate(5276, world, ms_max / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"ms_max": ms_max, "rate": rate}, fh)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert got[0] == got[1]
    assert got[0]["ms_max"] == 15.0
    assert got[0]["rate"] == pytest.approx(2 * 5276 / 0.015)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(100, 1, 0.5) == 200.0
    assert bench.job_rate(100, 4, 0.5) == 800.0


def test_dist_env_and_reference_arm_on_other_ranks(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (2, 1, 1)

    class Args:
        workload, steps, warmup, ref_units = "batched_exact", 1, 0, 4
    assert bench.run_reference(Args()) is None      # rank 1: exits without work and prints nothing
    assert capsys.readouterr().out == ""
