"""The multi-rank path of bench.py (replicas: barrier, max-over-ranks time,
aggregate throughput) on two CPU processes with the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, size, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(size), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1101_2065_gb300.replicas import Replicas
    r = Replicas("gloo")
    r.barrier()
    elapsed = [100.0, 250.0][rank]          # rank 1 is the slow one
    out[rank] = (r.max(elapsed), r.throughput(5, elapsed))
    r.barrier()
    r.close()


def test_two_rank_replicas_gloo():
    size = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, size, port, out)) for i in range(size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank in range(size):
        t_max, thr = out[rank]
        assert t_max == 250.0
        assert thr == pytest.approx(2 * 5 / 0.25)


def test_single_rank_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_1101_2065_gb300.replicas import Replicas
    r = Replicas("gloo")
    assert (r.rank, r.size) == (0, 1)
    assert r.max(3.0) == 3.0
    assert r.throughput(4, 2000.0) == pytest.approx(2.0)
