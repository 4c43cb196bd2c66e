"""Replica (weak-scaling) host logic of bench.py on CPU with gloo, world size 2.

Each rank times its own factorisation; the job value is the flops of all
ranks over the slowest rank's time.  No GPU is used.
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]
    ms_max = bench.max_over_ranks(ms, world, device="cpu")
    bench.barrier(world)
    out[rank] = (ms_max, bench.job_value(1e9, world, ms_max))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert abs(res[0][1] - 2e9 / 0.150 / 1e9) < 1e-9


def test_reference_arm_nonzero_rank_exits(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
