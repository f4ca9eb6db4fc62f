"""The benchmark's multi-rank host logic at world size 2, on CPU with gloo.

Under torchrun every rank solves its own replica of a single-instance
workload (that solve does not shard), and the batched workload's one instance
list is split over the ranks by LPT on instance size.  Nothing on the data
path crosses ranks: the collectives are the max over ranks of the timings and
the gather of the per-pair statistics.  These tests check that the ranks'
seeded inputs differ, that the job time is the slowest rank's, the LPT
partition, the merged statistics, and that the reference arm runs on rank 0
only.
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
        seeds = {w: bench.replica_seed(w, 0, rank) for w in ("grf350", "blocks32")}
        timed = bench.max_over_ranks([10.0 + rank, 3.0 - rank], "cpu", world)
        k = I.workload_blocks32(seed=seeds["blocks32"], n=8)["kappa"]
        bt = I.workload_batched(seed=seeds["blocks32"] * 100, count=2, nrhs=1, lo=4, hi=6)
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


def test_lpt_partition_covers_balances_and_is_deterministic():
    import bench
    from paper_1909_09771_gb300 import inputs as I
    grids = I.batched_grids(seed=0, count=64 * 4)
    sizes = [g[0] * g[1] * g[2] for g in grids]
    for nranks in (1, 2, 3, 4, 8):
        parts = bench.lpt_partition(sizes, nranks)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))            # every instance exactly once
        loads = [sum(sizes[i] for i in p) for p in parts]
        # Graham's bound for LPT: no rank exceeds the mean by more than the largest instance
        assert max(loads) <= sum(loads) / nranks + max(sizes)
        assert parts == bench.lpt_partition(sizes, nranks)
    # a hand case, sizes 7, 5, 4, 3, 1 over two ranks, in LPT order: 7 -> rank 0 (loads 7, 0),
    # 5 -> rank 1 (7, 5), 4 -> rank 1 (7, 9), 3 -> rank 0 (10, 9), 1 -> rank 1 (10, 10)
    assert bench.lpt_partition([7, 5, 4, 3, 1], 2) == [[0, 3], [1, 2, 4]]


def test_batched_generator_indices_match_full_list():
    from paper_1909_09771_gb300 import inputs as I
    full = I.workload_batched(seed=3, count=6, nrhs=2, lo=4, hi=7)
    part = I.workload_batched(seed=3, count=6, nrhs=2, lo=4, hi=7, indices=[4, 1])
    assert [w["grid"] for w in full] == I.batched_grids(seed=3, count=6, lo=4, hi=7)
    for k, i in enumerate([4, 1]):
        assert part[k]["grid"] == full[i]["grid"]
        assert (part[k]["kappa"] == full[i]["kappa"]).all() and (part[k]["b"] == full[i]["b"]).all()


def _lpt_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1909_09771_gb300 import inputs as I
        count, nrhs = 10, 3
        grids = I.batched_grids(seed=0, count=count, lo=4, hi=9)
        mine = bench.lpt_partition([g[0] * g[1] * g[2] for g in grids], world)[rank]
        # stand-in per-pair stats: what each rank's batched solve would report
        local = [{"pair": i * nrhs + j, "rank": rank} for i in mine for j in range(nrhs)]
        merged = bench.merge_pair_stats(local, mine, nrhs, count, world)
        q.put((rank, mine, merged))
    finally:
        dist.destroy_process_group()


def test_two_ranks_lpt_shards_and_merged_stats():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            rank, mine, merged = q.get(timeout=180)
            out[rank] = (mine, merged)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    m0, m1 = out[0][0], out[1][0]
    assert sorted(m0 + m1) == list(range(10)) and not set(m0) & set(m1)
    for rank in (0, 1):
        merged = out[rank][1]
        assert [s["pair"] for s in merged] == list(range(30))   # global pair order
        for s in merged:
            assert s["rank"] == (0 if s["pair"] // 3 in m0 else 1)
