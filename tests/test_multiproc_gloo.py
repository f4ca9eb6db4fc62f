"""The benchmark's multi-rank host logic at world size 2, on CPU with gloo.

Under torchrun every rank solves its own replica (the single-instance solve
does not shard; the batched workload's instances are independent), with no
collective on the data path: the only collective is the max over ranks of the
timings.  These tests check that the ranks' seeded inputs differ, that the job
time is the slowest rank's, and that the reference arm runs on rank 0 only.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1909_09771_gb300 import inputs as I
        seeds = {w: bench.replica_seed(w, 0, rank) for w in ("grf350", "blocks32", "batched")}
        timed = bench.max_over_ranks([10.0 + rank, 3.0 - rank], "cpu", world)
        k = I.workload_blocks32(seed=seeds["blocks32"], n=8)["kappa"]
        bt = I.workload_batched(seed=seeds["batched"], count=2, nrhs=1, lo=4, hi=6)
        fp = torch.tensor([float(k.sum()), float(bt[0]["kappa"].sum()), float(bt[1]["b"].sum())],
                          dtype=torch.float64)
        every = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(every, fp)
        q.put((rank, seeds, timed, [t.tolist() for t in every]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_distinct_replicas_and_slowest_rank_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            rank, seeds, timed, every = q.get(timeout=180)
            out[rank] = (seeds, timed, every)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(out) == [0, 1]
    for rank in (0, 1):
        seeds, timed, every = out[rank]
        assert timed == [11.0, 3.0]                  # max over ranks, element-wise
        assert every[0] != every[1]                  # the two replicas are different problems
        assert every[0][0] != every[1][0] and every[0][1] != every[1][1]
    # batched replicas span disjoint seed ranges (one seed per instance, 64 instances)
    s0, s1 = out[0][0]["batched"], out[1][0]["batched"]
    assert abs(s1 - s0) >= 64
    assert out[0][0]["grf350"] != out[1][0]["grf350"]


def test_single_rank_max_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], "cpu", 1) == [1.5, 2.5]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload = "blocks32"
        seed = 0
        warmup = 3
        steps = 1
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
