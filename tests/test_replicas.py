"""Multi-GPU host logic of bench.py (replicas, no collective on the data path),
run as world_size-2 gloo process groups on CPU: the rank-rotated roots, the
max-over-ranks timed region and the whole-job aggregate; and the reference arm
doing no work off rank 0."""
import os
import socket

import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        roots = bench.replica_roots(list(range(10, 74)), rank)
        local_ms = 100.0 + 25.0 * rank            # rank 1 is the slower replica
        total = bench.max_over_ranks(local_ms, ws, device="cpu")
        out.put((rank, roots[0], sorted(roots) == list(range(10, 74)), total,
                 bench.aggregate_gteps(ws, 16, 10**9, total)))
    finally:
        dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, first0, full0, t0, v0), (r1, first1, full1, t1, v1) = res
    assert (r0, r1) == (0, 1)
    assert first0 != first1                      # replicas start from different roots
    assert full0 and full1                       # each rank still cycles through every root
    assert t0 == t1 == 125.0                     # the job's time is the slowest rank's
    assert v0 == v1 == pytest.approx(2 * 16 * 10**9 / 0.125 / 1e9)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.replica_roots([1, 2, 3], 0) == [1, 2, 3]
    assert bench.replica_roots([1, 2, 3], 4) == [2, 3, 1]


def test_reference_arm_off_rank0_does_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"workload": "rmat", "layout": "csr", "mode": "do", "steps": 1, "warmup": 3,
                          "scale": 26, "cpu_scale": 22})()
    assert bench.reference_arm(args) == 0
    assert capsys.readouterr().out == ""


def test_served_capacity_criterion_uses_the_traces_own_rate():
    """A Poisson trace of k queries at nominal rate r spans (k-1)/r only on average: a server
    that kept pace with a trace that ran long must not be judged slow against r."""
    import numpy as np
    rng = np.random.default_rng(3)
    rate, k = 400.0, 1000
    arr = np.cumsum(rng.exponential(1.0 / rate, k))
    arr -= arr[0]
    realized = (k - 1) / arr[-1]
    # served exactly at the trace's pace, p99 well under half the target: keeps pace
    assert bench.keeps_pace(arr, realized, 30.0, 100.0)
    # a trace that happened to span 5 % longer than average is still kept pace with
    long_arr = arr * 1.05
    assert bench.keeps_pace(long_arr, (k - 1) / long_arr[-1], 30.0, 100.0)
    assert not (k - 1) / long_arr[-1] >= 0.97 * rate   # the nominal-rate test would have failed it
    # falling behind the trace, or a tail over half the target, does not keep pace
    assert not bench.keeps_pace(arr, 0.9 * realized, 30.0, 100.0)
    assert not bench.keeps_pace(arr, realized, 60.0, 100.0)
