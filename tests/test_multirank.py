"""World-size-2 gloo checks of the host-side multi-GPU logic (no GPU needed):
sharding covers every pulse exactly once, the step time reduces to the
maximum over ranks, and peak records gather in rank order."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    from paper_cs_0607001_gb300 import multigpu as M
    r, w, _ = M.init("gloo")
    assert (r, w) == (rank, world)
    lo, hi = M.shard(4097, r, w)
    M.barrier()
    t = M.max_over_ranks(1.5 + r)
    s = M.sum_over_ranks(hi - lo)
    rows = M.gather_rows([(r, lo, hi)], w)
    q.put((r, lo, hi, t, s, rows))
    dist.destroy_process_group()


def test_shard_partitions_exactly():
    from paper_cs_0607001_gb300 import multigpu as M
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            spans = [M.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.timeout(120)
def test_two_rank_gloo_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=90) for _ in range(2)])
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, lo0, hi0, t0, s0, rows0), (r1, lo1, hi1, t1, s1, rows1) = res
    assert (lo0, hi0, lo1, hi1) == (0, 2049, 2049, 4097)
    assert t0 == t1 == 2.5
    assert s0 == s1 == 4097
    assert rows0 == rows1 == [[(0, 0, 2049)], [(1, 2049, 4097)]]
