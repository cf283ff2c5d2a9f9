"""The multi-rank (torchrun) path of bench.py on CPU: two gloo ranks.

Each rank draws its own samples (weak scaling, no data-path collective); the
only collectives are the reductions of the timing report: the units of all
ranks are summed and divided by the slowest rank's time.  Also: the
reference arm runs on rank 0 alone.
"""
import argparse
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, tmp):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle import oracle as orc
        Lx = Ly = 4
        N, n = Lx * Ly, 6
        s = bench.rank_samples(rank, n, Lx, Ly)
        _, entries, _ = orc.connected(0, Lx, Ly, False, s)
        logical = n * N + len(entries) * N
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        rate, ms_max = bench.whole_job_rate(logical, ms, world, torch.device("cpu"))
        np.savez(os.path.join(tmp, f"rank{rank}.npz"), s=s, logical=logical, rate=rate,
                 ms_max=ms_max)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_samples_and_reduce_timing(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # each rank has its own zero-magnetisation samples
    assert not np.array_equal(r[0]["s"], r[1]["s"])
    for k in range(world):
        assert np.all(r[k]["s"].sum(axis=1) == 8)
    # every rank reports the same whole-job numbers: summed units / slowest time
    total = int(r[0]["logical"]) + int(r[1]["logical"])
    for k in range(world):
        assert float(r[k]["ms_max"]) == 15.0
        assert abs(float(r[k]["rate"]) - total / 0.015) <= 1e-9 * total / 0.015


def test_single_rank_reduction_is_identity():
    import bench
    rate, ms = bench.whole_job_rate(1000, 250.0, 1, None)
    assert ms == 250.0 and rate == 4000.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(workload="heisenberg_52x52", steps=1, warmup=3, gpus=2,
                              cpu_seconds=15.0)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
