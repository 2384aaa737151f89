"""Multi-process host logic of the replica runs (one process per GPU), on CPU
with the gloo backend and world size 2: the barrier and max-over-ranks that
bracket the timed region, and the model shards of a batched run."""
import os
import socket

import pytest

from paper_2608_23245_b300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    r, w = replicas.dist_init("gloo")
    assert (r, w) == (rank, world)
    replicas.barrier(w)
    mx = replicas.max_over_ranks(1.5 + rank, w, "cpu")
    tot = replicas.sum_over_ranks(float(rank + 1), w, "cpu")
    b, e = replicas.shard_range(256, r, w)
    units = replicas.sum_over_ranks(float(e - b), w, "cpu")
    out.put((rank, mx, tot, b, e, units))
    dist.destroy_process_group()


def test_gloo_world2_barrier_max_and_shards():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [2.5, 2.5]           # max over ranks
    assert [r[2] for r in res] == [3.0, 3.0]           # sum over ranks
    assert res[0][3:5] == (0, 128) and res[1][3:5] == (128, 256)
    assert [r[5] for r in res] == [256.0, 256.0]      # units processed by all ranks


@pytest.mark.parametrize("n,world", [(0, 3), (1, 4), (7, 2), (256, 8), (255, 8), (1000, 7)])
def test_shard_range_partitions(n, world):
    spans = [replicas.shard_range(n, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (b0, e0), (b1, e1) in zip(spans, spans[1:]):
        assert e0 == b1
    sizes = [e - b for b, e in spans]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_shard_range_rejects_bad_input():
    with pytest.raises(ValueError):
        replicas.shard_range(10, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard_range(-1, 0, 1)
