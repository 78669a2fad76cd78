"""The multi-rank path (replicas, no data exchange) with world size 2 on CPU (gloo)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2305_07253_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    assert replicas.init("gloo")
    r, w, _ = replicas.env()
    replicas.barrier()
    mx = replicas.max_over_ranks(1.5 + r)
    sm = replicas.sum_over_ranks(10.0 * (r + 1))
    b, e = replicas.shard(1001, r, w)
    out.put((r, mx, sm, b, e))
    replicas.finalize()


def test_two_ranks_agree_on_max_sum_and_cover_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [2.5, 2.5]      # max of 1.5 and 2.5 on both ranks
    assert [x[2] for x in res] == [30.0, 30.0]
    assert res[0][3:] == (0, 501) and res[1][3:] == (501, 1001)


def test_single_process_is_a_no_op():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.shard(10, 0, 1) == (0, 10)
    with pytest.raises(AssertionError):
        assert replicas.init("gloo")  # world size 1: no group
