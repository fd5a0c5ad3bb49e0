"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the
instance shards are disjoint, the step time is the slowest rank's, and the
rate counts every rank's precoders.  The GPU kernels are not involved."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, times, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard(rank, n)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    slowest = bench.max_over_ranks(times[rank], dist, "cpu")
    rate = bench.whole_job_rate(n, world, slowest)
    out[rank] = (gathered, slowest, rate)
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world, n = 2, 5
    times = [12.5, 20.0]
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, n, times, out), nprocs=world, join=True)
        res = dict(out)
    import bench
    for rank in range(world):
        gathered, slowest, rate = res[rank]
        flat = [i for g in gathered for i in g]
        assert sorted(flat) == list(range(world * n))  # disjoint and complete
        assert slowest == max(times)
        assert rate == pytest.approx(n * bench.NRHS * world / (max(times) / 1000.0))


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
