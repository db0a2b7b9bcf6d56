"""The benchmark's multi-rank host logic (replicas only: no data-path
collective) on two CPU processes over gloo: rates are whole-job figures (the
units of all ranks, summed) over the slowest rank, every mode table is
reduced the same way on every rank, each rank packs its own seeded workload,
and the reference arm runs on rank 0 alone."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        t = [2.0, 5.0][rank]
        rate = bench.job_rate(1000.0, t, world)
        # ranks whose seeded workloads differ in size: units are summed
        rate_uneven = bench.job_rate([1000.0, 400.0][rank], t, world)
        slow = bench.max_over_ranks([0.3, 0.1][rank], world)
        extra = {"fp64": {"value": 100.0 / [1.0, 4.0][rank], "ms_per_step": [1.0, 4.0][rank]},
                 "echem": {"config": {"workload": "x"},
                           "a": {"value": 10.0, "ms_per_step": [2.0, 3.0][rank]},
                           "b": {"value": 7.0, "ms_per_step": 1.5}},
                 "ratio": 3.0}
        bench.reduce_modes(extra, world)
        q.put((rank, rate, rate_uneven, slow, extra))
    finally:
        dist.destroy_process_group()


def test_rates_over_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, rate, rate_uneven, slow, extra = q.get(timeout=120)
        out[rank] = (rate, rate_uneven, slow, extra)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        rate, rate_uneven, slow, extra = out[rank]
        assert rate == pytest.approx(2 * 1000.0 / 5.0)
        assert rate_uneven == pytest.approx((1000.0 + 400.0) / 5.0)
        assert slow == pytest.approx(0.3)
        # fp64: rank 0 ran 100 units at 1 ms, rank 1 at 4 ms -> 2 x 100 units / 4 ms
        assert extra["fp64"]["ms_per_step"] == pytest.approx(4.0)
        assert extra["fp64"]["value"] == pytest.approx(2 * 100.0 / 4.0)
        assert extra["echem"]["a"]["ms_per_step"] == pytest.approx(3.0)
        # units per step of each rank (value x ms) summed over the slowest rank's ms
        assert extra["echem"]["a"]["value"] == pytest.approx((10.0 * 2.0 + 10.0 * 3.0) / 3.0)
        assert extra["echem"]["b"]["value"] == pytest.approx(14.0)
        assert extra["ratio"] == 3.0


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(0.7, 1) == 0.7
    assert bench.job_rate(50.0, 2.0, 1) == 25.0
    extra = {"m": {"value": 3.0, "ms_per_step": 2.0}}
    bench.reduce_modes(extra, 1)
    assert extra == {"m": {"value": 3.0, "ms_per_step": 2.0}}


def test_each_rank_packs_its_own_workload():
    import numpy as np
    import bench
    s0, g0 = bench.workload("c1", 0)
    s1, g1 = bench.workload("c1", 1)
    assert s1.seed == s0.seed + 1000
    assert g0["a"].shape == g1["a"].shape
    assert not np.array_equal(g0["x"], g1["x"])


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import sys
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                      "--warmup", "0", "--workload", "c1"])
    args = bench.parse()
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
