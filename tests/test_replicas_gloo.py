"""Host logic of the multi-GPU bench on CPU: two gloo ranks (world size 2).

The solve does not shard (one PCG per GPU, no data-path collective), so `bench.py --gpus N`
runs N independent replicas. What the ranks share is host logic: the timed region ends with
the slowest replica (max over ranks), and the reference arm runs on rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # per-rank elapsed times: every rank gets the slowest one
        got = bench.max_over_ranks(1.25 + rank, dist, "cpu")
        # the reference arm: ranks other than 0 exit at once with status 0 and no work
        class Args:
            workload = bench.DEFAULT_WORKLOAD
            steps = 1
            warmup = 0
            ref_iterations = 877
            loads = "traction"
            blocks = "vertex"
            eta_bar = 1.0
        ref = bench.run_reference(Args, rank, world) if rank != 0 else 0
        out.put((rank, got, ref))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_and_reference_runs_on_rank_0_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2.25, 2.25]
    assert [r[2] for r in res] == [0, 0]


def test_max_over_ranks_without_process_group_is_the_value():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
