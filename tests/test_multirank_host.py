"""Host logic of the multi-GPU benchmark path, on CPU with two gloo ranks.

The gradient workload does not shard across GPUs in the library: N GPUs run N
independent replicas (one seeded design per rank, no data-path collective),
timed by the slowest rank.  These tests run the benchmark's rank helpers
under a real two-process gloo group: the max-over-ranks reduction, the
whole-job rate, the per-rank workloads, and the reference arm that only
rank 0 runs.
"""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    import bench
    cpu = torch.device("cpu")
    got_ws, got_rank, _ = bench.dist_env()
    # each rank "timed" a different duration; all must see the slowest
    t = bench.max_over_ranks(1.5 + rank, ws, cpu)
    w = bench.workload(rank, n_steps=7)
    dist.barrier()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([got_ws, got_rank, t, w.n_cells, w.n_steps, float(w.eps.sum())]))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_run_own_designs(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    r = [np.load(tmp_path / f"rank{i}.npy") for i in range(ws)]
    for i, v in enumerate(r):
        assert v[0] == ws and v[1] == i
        assert v[2] == 1.5 + (ws - 1)          # max over ranks, seen by every rank
        assert v[3] == r[0][3] and v[4] == 7   # same shape and step count
    assert r[0][5] != r[1][5]                  # but an independent design per rank


def test_job_rate_is_whole_job_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.job_rate(1, 4_000_000 * 2000, 5, 2.0)
    assert one == pytest.approx(4e6 * 2000 * 5 / 2.0 / 1e9)
    # N replicas in the same (slowest-rank) time: N times the throughput
    assert bench.job_rate(4, 4_000_000 * 2000, 5, 2.0) == pytest.approx(4 * one)
    assert bench.max_over_ranks(3.25, 1, None) == 3.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_step", lambda n: called.append(n))
    args = type("A", (), dict(cpu_sample_steps=4, warmup=3, steps=1))()
    bench.run_reference(args)
    assert called == [] and capsys.readouterr().out == ""
