"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2).

Each rank evaluates its own independent system (weak scaling); the job time
is the slowest rank's and the throughput counts every rank's atoms.  No GPU
and no collective in the data path: only the timing all-reduce.
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


def _worker(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, tmax = bench.aggregate(times[rank], atoms_per_rank=4096, steps=10, dist=dist, device="cpu")
        q.put((rank, value, tmax))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(1.0, 2.0), (0.5, 0.25)])
def test_weak_scaling_aggregate_over_two_gloo_ranks(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tmax = max(times)
    for rank, value, t in out:
        assert t == pytest.approx(tmax)
        assert value == pytest.approx(4096 * 2 * 10 / tmax)


def test_single_rank_aggregate():
    import bench
    value, t = bench.aggregate(2.0, atoms_per_rank=4096, steps=10, dist=None, device="cpu")
    assert t == 2.0 and value == pytest.approx(4096 * 10 / 2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm runs (and prints) on rank 0 only."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "reference_arm", lambda args: called.append(args))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    bench.main()
    assert called == [] and capsys.readouterr().out == ""
