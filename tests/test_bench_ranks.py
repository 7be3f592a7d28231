"""Host logic of the multi-rank bench on CPU: world size 2 over gloo
(127.0.0.1).  Every rank gets the slowest rank's step time, the whole-job
throughput counts all ranks' unknowns against it (weak scaling), and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        step = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
        dist.barrier()
        out[rank] = step
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}
    # 2 ranks x 2,097,152 unknowns in 15 ms
    assert abs(bench.job_mdof_s(2097152, ws, 15.0) - 2 * 2097152 / 15e-3 / 1e6) < 1e-9


def test_one_rank_is_the_plain_value():
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert abs(bench.job_mdof_s(1000, 1, 2.0) - 0.5) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps = 1
        warmup = 0
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
