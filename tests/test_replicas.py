"""Multi-rank host logic on CPU (gloo, world size 2): sharding of the fills
and the whole-job throughput (units of all ranks over the slowest rank's
time).  No GPU and no data-path collective are involved."""
import os
import socket

import pytest

from paper_1611_04959_gb300 import replicas


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (7, 2), (24, 4), (16, 3), (1152, 8)])
def test_shards_cover_every_unit_once(n, world):
    seen = []
    sizes = []
    for r in range(world):
        s = replicas.shard(n, r, world)
        seen += list(s)
        sizes.append(len(s))
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_arguments():
    for args in [(5, 2, 2), (5, -1, 2), (5, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            replicas.shard(*args)


def test_aggregate_without_process_group():
    b, ms, gbs = replicas.aggregate(2e9, 1000.0)
    assert (b, ms) == (2e9, 1000.0) and gbs == pytest.approx(2.0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        fills = list(replicas.shard(48, rank, world))
        replicas.barrier()
        # rank r "processed" its fills in (10 + 5 r) ms
        tot, mx, gbs = replicas.aggregate(len(fills) * 1.45e9, 10.0 + 5.0 * rank)
        replicas.barrier()
        q.put((rank, fills, tot, mx, gbs))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == list(range(24)) and out[1][1] == list(range(24, 48))
    for _, _, tot, mx, gbs in out:
        assert tot == pytest.approx(48 * 1.45e9)
        assert mx == 15.0                       # the slowest rank's time
        assert gbs == pytest.approx(48 * 1.45e9 / 15e-3 / 1e9)
