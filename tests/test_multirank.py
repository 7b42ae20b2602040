"""The host logic of bench.py's N-rank runs (one replica per rank; the path does
not shard), on CPU with the gloo backend and two ranks: the max-over-ranks time,
the whole-job throughput, rank detection, and the reference arm that only rank 0
runs."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench._env_rank()
        # every rank times something different; all of them see the slowest
        t = bench._max_over_ranks(1.5 + 2.0 * rank, dist, device="cpu")
        dist.barrier()
        out[rank] = (r, w, lr, t, bench._throughput(w, 1000, 10, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, lr, t, v) in res.items():
        assert (r, w, lr) == (rank, world, rank)
        assert t == 3.5  # the slower rank's time, on every rank
        assert v == pytest.approx(world * 1000 * 10 / 3.5)


def test_single_rank_needs_no_process_group():
    assert bench._max_over_ranks(2.25, None) == 2.25
    assert bench._throughput(1, 2097152, 10, 0.05) == pytest.approx(2097152 * 10 / 0.05)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(None) is None  # returns before any work
    assert buf.getvalue() == ""
