"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) run bench.py's
rank bookkeeping and max-over-ranks reduction; every rank must see the
slowest rank's times and the weak-scaling throughput of the whole job."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, local = bench._dist()
    # rank r's device and end-to-end step times
    dev_s, e2e_s = bench.reduce_max([1.0 + 0.5 * r, 3.0 - r], dist)
    dist.barrier()
    q.put((r, w, local, dev_s, e2e_s, bench.job_throughput(w, dev_s)))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, local, dev_s, e2e_s, bps in out:
        assert w == 2 and local == r
        assert dev_s == 1.5 and e2e_s == 3.0          # the slowest rank's times
        assert abs(bps - 2 / 1.5) < 1e-12              # two bodies per step of the slowest rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([0.25, 4.0]) == [0.25, 4.0]
    assert bench.job_throughput(1, 0.5) == 2.0
