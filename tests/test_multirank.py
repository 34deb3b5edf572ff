"""The multi-rank logic of bench.py on CPU (gloo, world size 2).  Every rank
runs its own instance (replicas: no collective on the data path); the job's
time is the slowest rank's, its throughput the units of all ranks over that
time, and the reference arm runs on rank 0 only."""
import os
import socket
import types

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ws, r, local = bench.dist_env()
    ms = bench.max_over_ranks(torch, [12.5, 20.0][rank], ws, device="cpu")
    value = bench.job_value(1000, ws, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ws, r, local, ms, value))


def test_two_ranks_report_the_slowest_time_and_the_whole_job():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, (r, ws, rr, local, ms, value) in enumerate(res):
        assert (r, ws, rr, local) == (rank, 2, rank, rank)
        assert ms == 20.0  # both ranks see the slower rank's time
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, {"name": "unused"}) is None
    assert capsys.readouterr().out == ""
