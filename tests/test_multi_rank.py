"""The benchmark's multi-rank path (one replica per rank; the job's time is
the slowest rank's) with two gloo ranks on the CPU: the max over ranks, the
whole-job rate, and that only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(100.0 + 25.0 * rank)   # this rank's total ms
        rate = bench.job_rate(world, 2_000_000, 10, slowest)
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in got:
        assert slowest == 125.0                      # both ranks see the slowest rank
        assert rate == pytest.approx(2 * 2_000_000 * 10 / 0.125)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 100, 2, 1000.0) == pytest.approx(200.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    a = bench.parse()
    a.theta = 0.7
    assert bench.reference_arm(a) is None
    assert capsys.readouterr().out == ""


def test_committed_walk_profiles_match_the_sources():
    """The ncu summaries the benchmark takes its DRAM traffic from are of the
    walk sources as they are now (their recorded hash), for the benchmark's
    workloads; any other workload or mode gets no traffic figure."""
    import bench
    w = "maclaurin_e0.9_L2+3"
    assert bench.captured_traffic(w, 0.75, "quadrupole") is not None
    assert bench.captured_traffic(w, 0.72, "quadrupole") is None
    assert bench.captured_traffic(w, 0.7, "periodic64") is not None
    assert bench.captured_traffic(w, 0.7, "quadrupole") is None
    assert bench.captured_traffic(w, 0.24, "monopole") is not None
    assert bench.captured_traffic(bench.BATCH_WORKLOAD, 0.5, "batched_monopole") is not None
    assert bench.captured_traffic(bench.BATCH_WORKLOAD, 0.7, "batched_monopole") is None
    assert bench.captured_traffic(w, 0.72, "monopole") is None
    assert bench.captured_traffic("cloud_core", 0.72, "quadrupole") is None
