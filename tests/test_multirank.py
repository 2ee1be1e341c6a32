"""The multi-rank timing path of bench.py on CPU ranks (gloo, world size 2):
every rank gets the slowest rank's time, and the reported value counts the
pixels of all ranks (weak scaling: one independent pair per rank)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        got = bench.max_over_ranks(ms, ws, device=None)
        value = bench.whole_job_value(1000, ws, 4, got)
        out[rank] = (got, value)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 15.0
    # 2 ranks x 1000 px x 4 steps in 15 ms
    assert abs(out[0][1] - 2 * 1000 * 4 / 0.015 / 1e6) < 1e-12
    assert out[0][1] == out[1][1]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert abs(bench.whole_job_value(8294400, 1, 10, 56.2 * 10) - 147.59) < 0.05
