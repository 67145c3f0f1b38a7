"""The replicated (N > 1) bench path's host logic on CPU: two gloo ranks,
whole-job time = slowest rank, units = sum over ranks, and a reference arm
that only rank 0 runs."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms, units = b.reduce_over_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), world, "cpu")
        out[rank] = (ms, units)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_summed_units():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    for r in range(world):
        assert got[r] == (15.0, 300.0)


def test_single_rank_is_identity():
    b = _bench()
    assert b.reduce_over_ranks(3.5, 7.0, 1, "cpu") == (3.5, 7.0)


def test_reference_arm_skips_non_zero_ranks(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:  # the reference arm must return before touching the workload
        workload = "c3"
    b.run_reference(A())
    assert capsys.readouterr().out == ""
