"""Host logic of the multi-GPU bench path on CPU: two gloo ranks (replicas)
take disjoint source ranges, the job time is the slowest rank's, throughput
counts every rank's solves; the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        base = bench.replica_source_base(rank, 16, 7)
        t = bench.max_over_ranks(dist, 1.5 + rank)  # rank 1 is the slower one
        q.put((rank, base, t, bench.job_throughput(16, 4, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, b0, t0, v0), (r1, b1, t1, v1) = res
    assert (r0, r1) == (0, 1)
    assert b0 == 0 and b1 == 16 * 7  # disjoint source ranges of 16 x 7 sources
    assert t0 == t1 == 2.5  # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(16 * 4 * 2 / 2.5)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(None, 3.25) == 3.25
    assert bench.job_throughput(16, 4, 1, 2.0) == 32.0


def test_reference_arm_only_on_rank_zero(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"workload": "c2", "warmup": 0, "steps": 1, "gpus": 2})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, dict(bench.WORKLOADS["c2"]))
    assert buf.getvalue() == ""


def test_cpu_baseline_fields_one_and_all_cores():
    """The oracle CPU baseline (spawned single-threaded processes) reports the
    cores it used and the one-core figure beside the all-cores one."""
    w = dict(bench.WORKLOADS["c2"])
    r = bench.cpu_baseline(w, 100, budget_slices=1, procs=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["unit"] == "solves/s"
    assert r["one_core"]["cores"] == 1 and r["one_core"]["value"] > 0 and r["value"] > 0
    assert "1x16x16x16" in r["sample"]
