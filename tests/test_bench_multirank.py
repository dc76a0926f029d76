"""The N > 1 path of bench.py on the CPU: two gloo ranks (replicas) reduce their
step times to the maximum, and the whole-job throughput counts every rank's
solves against the slowest rank's time."""
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


def _rank(rank, ws, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    assert bench._dist() == (ws, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 100.0 + 50.0 * rank            # rank 1 is the slower replica
        ms_max = bench.max_over_ranks(local_ms, torch.device("cpu"), dist, ws)
        out[rank] = (ms_max, bench.replica_throughput(ws, 4, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_to_the_slowest_rank():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
        got = dict(out)
    assert got[0] == got[1]
    ms_max, value = got[0]
    assert ms_max == 150.0
    assert abs(value - ws * 4 / 0.150) < 1e-9


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu"), None, 1) == 12.5
    assert bench.replica_throughput(1, 20, 200.0) == 100.0
