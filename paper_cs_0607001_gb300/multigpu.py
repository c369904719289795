"""Host-side helpers for running the correlation on several GPUs of one node.

Pairs of (received pulse, stored reference) are independent, so a multi-GPU
run splits one batch across ranks: every rank stores the same references,
correlates its share of the pulses, and the peak records are gathered back in
batch order.  There is no collective on the data path; the only exchanges are
host-level: a barrier, the maximum of the per-rank step times, and the gather
of the peak records (about 16 bytes per pulse and scale).
"""
from __future__ import annotations

import os

import numpy as np

import torch
import torch.distributed as dist


def dist_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (1 rank if unset)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init(backend: str | None = None) -> tuple[int, int, int]:
    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world, local


def barrier():
    if dist.is_initialized():
        if dist.get_backend() == "nccl":
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def max_over_ranks(x: float) -> float:
    if not dist.is_initialized():
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    if not dist.is_initialized():
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) share of n units for `rank` (sizes differ by at most 1)."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_rows(rows, world: int):
    """All-gather a per-rank list/array of peak records (host objects) in rank order."""
    if not dist.is_initialized() or world == 1:
        return [rows]
    out = [None] * world
    dist.all_gather_object(out, rows)
    return out


def shard_by_cost(costs, world: int) -> list[np.ndarray]:
    """Split items of uneven cost over `world` ranks: largest first, each to
    the rank with the least total so far (ties to the lower rank).  Returns
    each rank's item indices in increasing order."""
    costs = np.asarray(costs, dtype=np.float64)
    load = np.zeros(world)
    owner = np.empty(len(costs), dtype=np.int64)
    for i in np.argsort(-costs, kind="stable"):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return [np.nonzero(owner == r)[0] for r in range(world)]


def subset_ragged(batch: dict, idx) -> dict:
    """The items `idx` of a packed ragged batch (keys refs and y: packed
    complex samples; offsets, N, J, filter, delays: per item), repacked in
    that order with offsets from 0 (even when every N is)."""
    idx = np.asarray(idx, dtype=np.int64)
    off, n = np.asarray(batch["offsets"]), np.asarray(batch["N"])
    seg = [np.arange(off[i], off[i] + n[i]) for i in idx]
    cat = np.concatenate(seg) if seg else np.zeros(0, np.int64)
    out = dict(batch)
    out["refs"], out["y"] = batch["refs"][cat], batch["y"][cat]
    for k in ("N", "J", "filter", "delays"):
        out[k] = np.asarray(batch[k])[idx]
    out["offsets"] = np.concatenate([[0], np.cumsum(n[idx])[:-1]]).astype(np.int64)
    return out


def pair_cost(N, J) -> np.ndarray:
    """Algorithmic flops of the all-lag, all-scale correlation of one pair:
    8 N^2 (2 - 2^-J) (N lags at each of the J + 1 scales)."""
    N = np.asarray(N, dtype=np.float64)
    J = np.asarray(J, dtype=np.float64)
    return 8.0 * N * N * (2.0 - 2.0 ** -J)


def gather_slots(index, counts, lag, mag, norm, n_items: int, world: int):
    """Gather the peak records of a split batch in batch order.

    This rank correlated the items `index` (positions in the whole batch, in
    the order its records are packed); item index[k] has counts[k] records
    (J + 1, one per scale).  Returns (lag, mag, norm) for all n_items items,
    packed by slot as a single-rank call would pack them (item i's scales at
    sum_{i' < i} (J_i' + 1)), on every rank."""
    index = np.asarray(index, dtype=np.int64)
    counts = np.asarray(counts, dtype=np.int64)
    mine = (index, counts, np.asarray(lag), np.asarray(mag), np.asarray(norm))
    parts = gather_rows(mine, world)
    cnt = np.zeros(n_items, dtype=np.int64)
    for idx, c, *_ in parts:
        cnt[idx] = c
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    total = int(cnt.sum())
    out_lag = np.full(total, -1, dtype=np.int32)
    out_mag = np.zeros(total, dtype=np.float32)
    out_norm = np.zeros(total, dtype=np.float64)
    seen = np.zeros(n_items, dtype=bool)
    for idx, c, lg, mg, nm in parts:
        src = np.concatenate([[0], np.cumsum(c)[:-1]]) if len(c) else np.zeros(0, np.int64)
        for k, i in enumerate(idx):
            if seen[i]:
                raise ValueError(f"item {int(i)} was correlated by two ranks")
            seen[i] = True
            out_lag[first[i]:first[i] + c[k]] = lg.reshape(-1)[src[k]:src[k] + c[k]]
            out_mag[first[i]:first[i] + c[k]] = mg.reshape(-1)[src[k]:src[k] + c[k]]
            out_norm[first[i]:first[i] + c[k]] = nm.reshape(-1)[src[k]:src[k] + c[k]]
    if not seen.all():
        raise ValueError(f"{int((~seen).sum())} items were correlated by no rank")
    return out_lag, out_mag, out_norm
