"""Ray-range sharding of one simulation across ranks (host-side merge).

Rays are independent until deduplication (Sec. II-B), so a launch can be
split into contiguous ray-id ranges, one per rank, with the scene
replicated.  Each rank simulates its range and reports, per path key, how
many of its candidates it validated (in ray-id order, the valid one
included) and its validated representative.  The merge replays the
single-run rule -- candidates in ray-id order (all of them, or at most
rep_tries when a cap is set), the first valid one represents the key --
over the shards in range order:

    budget = rep_tries
    for each shard in ray order holding the key:
        if the shard found a valid candidate within `budget` tries: take it
        else: budget -= tries; stop when the budget is spent

Because every shard tries its own candidates in ray-id order, a shard's
tries are a prefix of the global order restricted to its range, so the
merged representative and path are the single run's.  LOS paths (no
member rays) are the same on every shard.  Received power is then summed
over the merged paths per receiver; a sum of per-shard powers would count
keys found by several shards more than once.

The collective is an all-gather of each rank's summary (torch.distributed,
any backend); the merge itself is deterministic host code.
"""
from __future__ import annotations

import numpy as np

NO_REP = 0xFFFFFFFF


def shard_ranges(n_rays: int, world: int):
    """Contiguous ray-id ranges [lo, hi) of `world` shards."""
    edges = [(r * n_rays) // world for r in range(world + 1)]
    return [(edges[r], edges[r + 1]) for r in range(world)]


def summary(keys: dict, paths: dict) -> dict:
    """One shard's summary from Result.keys() and Result.paths():
    key -> (tried, rep ray id or NO_REP, path row or None)."""
    where = {(int(h), int(l)): i for i, (h, l) in enumerate(zip(paths["key_hi"], paths["key_lo"]))}
    out = {}
    for h, l, t, r in zip(keys["key_hi"], keys["key_lo"], keys["tried"], keys["rep"]):
        k = (int(h), int(l))
        out[k] = (int(t), int(r), {n: v[where[k]] for n, v in paths.items()} if k in where else None)
    # LOS paths: no candidates, identical on every shard
    for k, i in where.items():
        if k not in out:
            out[k] = (1, int(paths["rep"][i]), {n: v[i] for n, v in paths.items()})
    return out


def merge(summaries, rep_tries: int) -> dict:
    """Merge shard summaries (in ray-range order) into key -> (rep, path)."""
    keys = set()
    for s in summaries:
        keys.update(s.keys())
    out = {}
    for k in keys:
        budget = rep_tries if rep_tries > 0 else float("inf")  # 0: every candidate
        for s in summaries:
            if k not in s:
                continue
            tried, rep, path = s[k]
            if path is not None and tried <= budget:
                out[k] = (rep, path)
                break
            budget -= tried
            if budget <= 0:
                break
    return out


def merged_power(merged: dict, n_rx: int) -> np.ndarray:
    """Per-receiver power P_j = sum |a|^2 over the merged paths."""
    p = np.zeros(n_rx)
    for _, path in merged.values():
        a = np.asarray(path["a"], np.float64)
        p[int(path["rx"])] += float(a @ a)
    return p


def merge_distributed(local: dict, rep_tries: int, group=None) -> dict:
    """All-gather every rank's summary (rank order = ray-range order) and
    merge; every rank gets the same result."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    gathered = [None] * world
    dist.all_gather_object(gathered, local, group=group)
    return merge(gathered, rep_tries)
