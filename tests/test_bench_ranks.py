"""Host logic of bench.py's multi-rank launch (replicas, one per GPU), on CPU with
two gloo ranks: each rank reads its place from the torchrun environment, the
timed region's length is the maximum over ranks, and the reference arm runs on
rank 0 only."""

import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as td

    import bench

    td.init_process_group("gloo", rank=rank, world_size=world)
    info = bench.dist_info()
    t = bench.max_over_ranks(1.5 + rank, world, "cpu")  # rank r took 1.5 + r seconds
    td.barrier()
    td.destroy_process_group()
    q.put((rank, info, t))


def test_two_gloo_ranks_take_the_slowest_time():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [(0, 2, 0), (1, 2, 1)]
    assert [g[2] for g in got] == [2.5, 2.5]


def test_single_rank_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(0.3, 1, "cpu") == 0.3


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    ns = type("A", (), {"steps": 1, "warmup": 0})()
    assert bench.run_reference(ns, 1, 2) is None
    assert capsys.readouterr().out == ""


def test_both_arms_share_the_workload_keys():
    sys.path.insert(0, ROOT)
    import bench

    cfg = bench.workload_config([1104, 4512, 18240], 2)
    assert cfg["workload"] == bench.WORKLOAD and cfg["space_levels"] == [18240, 1104, 1104]
    assert bench.workload_config([1104, 4512, 18240, 73344], 1, "cfg2")["space_levels"] == [73344, 73344, 18240]
    assert cfg["parallelism"] == "replicas x2" and cfg["N"] == bench.N_STEPS
    json.dumps(cfg)
