"""Multi-rank path on CPU: batched patches split across ranks by cost (no data-path
collective) and the bench's max-over-ranks timing, run as two gloo processes."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1502_02935_gb300 import inputs, sharding


def test_partition_covers_every_patch_once_and_balances():
    cells = [s[0] ** 3 for s in inputs.blast_patch_specs(64, seed=1502)]
    for world in (1, 2, 4, 8):
        owned = sharding.partition(cells, world)
        flat = sorted(i for lst in owned for i in lst)
        assert flat == list(range(64))
        assert sharding.imbalance(cells, owned) < 1.25
    assert sharding.partition([5, 3], 4)[2:] == [[], []]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local, pg = bench.dist_setup()
    cells = [s[0] ** 3 for s in inputs.blast_patch_specs(64, seed=1502)]
    mine = sharding.partition(cells, w)[r]
    # ranks agree on the assignment without exchanging it; the only collective is the max
    t = bench.max_over_ranks(pg, float(10 + r))
    q.put((r, mine, t))
    pg.destroy_process_group()


def test_two_gloo_ranks_share_patches_and_reduce_time():
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
    (r0, m0, t0), (r1, m1, t1) = res
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    assert t0 == t1 == 11.0
