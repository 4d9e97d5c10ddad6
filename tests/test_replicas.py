"""The multi-GPU form of the bench is replicas only: every rank runs the whole
workload on its own GPU, and the host combines the ranks' timings.  These
tests run that host logic as two gloo ranks on the CPU: slowest-rank maxima,
one schedule chosen alike on every rank, and the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank 0 alone would pick "two streams" (0.9 ms), rank 1 alone "one stream";
        # the slowest-rank times are 1.2 / 1.5 / 1.1 ms: both must pick "staggered"
        ms = {"one stream": [1.0, 1.2][rank], "two streams": [0.9, 1.5][rank],
              "staggered": [1.1, 1.05][rank]}
        form = bench.choose_form(ms)
        worst = bench.max_over_ranks([float(rank + 1), 5.0 - rank, -1.0])
        out.put((rank, form, worst))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_schedule_and_maxima():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    assert [g[1] for g in got] == ["staggered", "staggered"]
    for _, _, worst in got:
        assert worst == [2.0, 5.0, -1.0]


def test_single_process_helpers():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks([3, 1.5]) == [3.0, 1.5]
    assert bench.choose_form({"a": 2.0, "b": 1.0, "c": 1.0}) == "b"
    # 4 replicas, each 2 * 4194304 points, slowest rank 0.5 ms per step
    assert bench.replica_value(2 * 4194304, 4, 0.5) == pytest.approx(6.7108864e10)


def test_reference_arm_runs_on_rank_zero_only():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    # the other ranks return before touching the oracle
    assert bench.run_reference(None, None, rank=1) is None
