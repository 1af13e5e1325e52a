"""Multi-rank host logic on CPU: shards of independent problems and the
whole-job throughput over two gloo ranks (no GPU)."""

import os

import pytest

from paper_1107_5719_gb300 import replicas as RP


def test_shard_covers_every_problem_once_and_balances():
    sizes = [274625] * 32 + [2146689] * 24 + [8520321] * 8
    ws = 4
    parts = [RP.shard(sizes, ws, r) for r in range(ws)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.05
    assert RP.shard(sizes, 1, 0) == list(range(len(sizes)))


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        RP.shard([1, 2], 2, 2)


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r "solved" r+1 problems in (r+1)*100 ms
        thr, ms = RP.weak_throughput(rank + 1, (rank + 1) * 100.0)
        out[rank] = (thr, ms)
    finally:
        dist.destroy_process_group()


def test_weak_throughput_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    # 3 problems in total, slowest rank 200 ms -> 15 problems/s on both ranks
    for r in range(2):
        thr, ms = out[r]
        assert ms == 200.0
        assert abs(thr - 15.0) < 1e-12


def test_single_process_is_identity():
    thr, ms = RP.weak_throughput(4, 500.0)
    assert ms == 500.0 and thr == 8.0


def _failing_worker(rank, ws, port, out):
    """Rank 1 fails on the host before the timing reduction and leaves;
    rank 0 must get an error from its collective within the group's
    timeout instead of waiting forever."""
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        out[rank] = "left"
        raise SystemExit(3)          # host-side failure: never joins the reduction
    try:
        RP.weak_throughput(1, 100.0)
        out[rank] = "no error"
    except Exception as e:           # gloo reports the lost peer or the timeout
        out[rank] = "error: " + type(e).__name__
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_rank_failure_surfaces_as_an_error():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3
    assert out[1] == "left"
    assert str(out[0]).startswith("error"), out[0]
    assert procs[0].exitcode == 0
