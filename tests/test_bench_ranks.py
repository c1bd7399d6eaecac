"""The bench's multi-rank path on the host: two gloo ranks (127.0.0.1) take the maximum of their
timed regions as the job's time and report the whole job's rate; the reference arm runs on
rank 0 only. No GPU: the collective is gloo on CPU tensors, as `bench.py --gpus N` does with
NCCL on the GPUs."""
import importlib.util
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    local = [0.75, 1.25][rank]
    s = b.job_seconds(local, world, device="cpu")
    out[rank] = (s, b.job_throughput(1000, world, s), b.dist_env()[:2])
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_rank():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in (0, 1):
        s, v, (rank, world) = out[r]
        assert s == 1.25 and world == 2 and rank == r
        assert v == pytest.approx(2 * 1000 / 1.25)


def test_single_rank_needs_no_collective():
    b = _bench()
    assert b.job_seconds(0.5, 1) == 0.5
    assert b.job_throughput(10, 1, 0.5) == 20


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert b.run_reference(None) is None      # returns before touching the oracle or args
    assert capsys.readouterr().out == ""
