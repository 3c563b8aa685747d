"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1), each timing its
own replica. The reported times are the slowest rank's, the throughput counts every rank's
cells, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # rank r "measured" (10 + r, 4 + 3 r, 12 - r) ms
    vals = torch.tensor([10.0 + rank, 4.0 + 3 * rank, 12.0 - rank], dtype=torch.float64)
    ms, fwd_ms, e2e_ms = bench.max_over_ranks(vals, ws)
    value = bench.job_throughput(1000, ws, ms)
    out[rank] = (ms, fwd_ms, e2e_ms, value, bench._dist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_all_cells():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        ms, fwd_ms, e2e_ms, value, d = res[rank]
        assert (ms, fwd_ms, e2e_ms) == (11.0, 7.0, 12.0)
        assert value == pytest.approx(1000 * ws / 11e-3)
        assert d == (ws, rank, rank)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    vals = torch.tensor([3.0, 4.0], dtype=torch.float64)
    assert bench.max_over_ranks(vals, 1) == [3.0, 4.0]
    assert bench.job_throughput(500, 1, 2.0) == pytest.approx(250000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "cpu_baseline_sample", lambda k: called.append(k))

    class Args:
        warmup, steps, gpus = 1, 1, 2
    bench.run_reference(Args())
    assert called == [] and capsys.readouterr().out == ""
