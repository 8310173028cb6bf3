"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2).

`bench.py --gpus N` runs one independent replica of the workload per rank
(the path shards by replicas, with no data-path collective); the timing is the
maximum over ranks and the value the whole job's throughput.  These tests run
that logic on two CPU processes: every rank receives the slowest time, the
aggregate counts both replicas, and the reference arm prints from rank 0 only.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.barrier_max(1.0 + rank, ws)          # rank 1 is the slower one
        env = bench.dist_env()
        q.put((rank, got, env, bench.aggregate_gdofs(1000, got, ws)))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, env, agg in res:
        assert got == 2.0                                  # the slowest rank's time everywhere
        assert env == (2, rank, rank)
        assert agg == pytest.approx(2 * 1000 / 2.0 / 1e9)  # both replicas over the max time


def test_single_rank_is_identity():
    assert bench.barrier_max(3.5, 1) == 3.5
    assert bench.aggregate_gdofs(16_777_216, 0.5e-3, 1) == pytest.approx(33.554432)


def test_reference_arm_prints_from_rank_zero_only(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 1, 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
