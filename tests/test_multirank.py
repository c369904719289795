"""World-size-2 gloo checks of the host-side multi-GPU logic (no GPU needed):
sharding covers every pulse exactly once, the step time reduces to the
maximum over ranks, and peak records gather in rank order."""
import os
import socket

import numpy as np
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


def _fake_records(items, Js):
    """Stand-in for a rank's correlation of its items: per item i and scale
    j a record that depends only on (i, j), packed in the order of `items`."""
    lag, mag, norm = [], [], []
    for i in items:
        for j in range(int(Js[i]) + 1):
            lag.append((37 * int(i) + 5 * j) % 1000)
            mag.append(float(i) + 0.25 * j)
            norm.append(1.0 / (1 + int(i) + j))
    return np.array(lag, np.int32), np.array(mag, np.float32), np.array(norm, np.float64)


def _ragged_list():
    g = np.random.default_rng(5)
    Ns = np.exp(g.uniform(np.log(256), np.log(65536), 301)).astype(np.int64) // 64 * 64
    Js = g.integers(3, 9, 301)
    return Ns, Js


def _split_worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    from paper_cs_0607001_gb300 import multigpu as M
    r, w, _ = M.init("gloo")
    # a uniform batch (4097 pulses, J = 5): contiguous shards
    B, J = 4097, 5
    Ju = np.full(B, J)
    lo, hi = M.shard(B, r, w)
    mine = np.arange(lo, hi)
    uni = M.gather_slots(mine, Ju[mine] + 1, *_fake_records(mine, Ju), B, w)
    # a ragged list: shards balanced by the pairs' correlation cost
    Ns, Js = _ragged_list()
    parts = M.shard_by_cost(M.pair_cost(Ns, Js), w)
    rag = M.gather_slots(parts[r], Js[parts[r]] + 1, *_fake_records(parts[r], Js), len(Ns), w)
    loads = [float(M.pair_cost(Ns[p], Js[p]).sum()) for p in parts]
    q.put((r, [a.tolist() for a in uni], [a.tolist() for a in rag], loads))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_split_batch_gathers_the_single_rank_records_in_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=90) for _ in range(2)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    B = 4097
    one_uni = _fake_records(np.arange(B), np.full(B, 5))
    Ns, Js = _ragged_list()
    one_rag = _fake_records(np.arange(len(Ns)), Js)
    for r, uni, rag, loads in res:
        for got, want in zip(uni, one_uni):
            np.testing.assert_array_equal(np.array(got), want)
        for got, want in zip(rag, one_rag):
            np.testing.assert_array_equal(np.array(got), want)
        assert max(loads) <= 1.05 * min(loads)  # cost-balanced shares


def test_gather_slots_rejects_overlap_and_gaps():
    from paper_cs_0607001_gb300 import multigpu as M
    Js = np.full(4, 2)
    rec = _fake_records(np.arange(4), Js)
    lag, mag, norm = M.gather_slots(np.arange(4), Js + 1, *rec, 4, 1)
    np.testing.assert_array_equal(lag, rec[0])
    with pytest.raises(ValueError, match="no rank"):
        M.gather_slots(np.arange(3), Js[:3] + 1, *_fake_records(np.arange(3), Js), 4, 1)
    with pytest.raises(ValueError, match="two ranks"):
        idx = np.array([0, 1, 1, 2, 3])
        M.gather_slots(idx, Js[idx] + 1, *_fake_records(idx, Js), 4, 1)


def test_subset_ragged_repacks_each_rank_share():
    """A rank's cost-balanced share of a ragged batch, repacked: every item's
    pulse and stored signal are the original samples, offsets start at 0 and
    stay even, and the shares together hold every item once."""
    from paper_cs_0607001_gb300 import inputs
    from paper_cs_0607001_gb300 import multigpu as M
    w = inputs.ragged_batch(n=240)
    parts = M.shard_by_cost(M.pair_cost(w["N"], w["J"]), 3)
    assert sorted(np.concatenate(parts).tolist()) == list(range(len(w["N"])))
    for idx in parts:
        s = M.subset_ragged(w, idx)
        assert s["offsets"][0] == 0 and (s["offsets"] % 2 == 0).all()
        assert len(s["y"]) == int(w["N"][idx].sum()) == len(s["refs"])
        for k, i in enumerate(idx):
            a, b = s["offsets"][k], w["offsets"][i]
            n = int(w["N"][i])
            assert s["N"][k] == n and s["J"][k] == w["J"][i] and s["filter"][k] == w["filter"][i]
            assert s["delays"][k] == w["delays"][i]
            np.testing.assert_array_equal(s["y"][a:a + n], w["y"][b:b + n])
            np.testing.assert_array_equal(s["refs"][a:a + n], w["refs"][b:b + n])
