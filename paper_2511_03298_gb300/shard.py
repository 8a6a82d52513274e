"""List-sharded search: the host side of the protocol (exchanges only).

Every arithmetic step runs in the library (ksc_shard_candidates,
ksc_shard_rerank, ksc_merge_topk); this module moves their outputs between
shards.  Two exchanges per search: the shards' candidate keys (so each shard
knows the whole index's R-th key) and their (distance, id) results.

  search_local(shards, ...)    several shards in one process (one device, or
                               one per device): the exchanges are stacks
  search_dist(shard, ...)      one shard per process: the exchanges are
                               torch.distributed all-gathers
"""


def owners_round_robin(sizes, parts):
    """A list partition that balances vectors: lists in decreasing size, each
    to the shard holding the fewest vectors so far (ties: lower shard)."""
    import numpy as np
    sizes = np.asarray(sizes)
    load = np.zeros(parts, np.int64)
    owner = np.zeros(len(sizes), np.int32)
    for p in np.argsort(-sizes, kind="stable"):
        g = int(np.argmin(load))
        owner[p] = g
        load[g] += int(sizes[p])
    return owner


def search_local(shards, Q, k, nprobe, rerank, opts=None, ip=False):
    """The sharded search with every shard in this process; Q on each shard's
    device is the caller's (shards on one device share it)."""
    import torch
    from . import ksc
    own = [s.shard_candidates(Q, k, nprobe, rerank, opts=opts) for s in shards]
    all_keys = torch.stack(own)
    res = [s.shard_rerank(Q, k, rerank, o, all_keys) for s, o in zip(shards, own)]
    ids = torch.stack([r[0] for r in res])
    dists = torch.stack([r[1] for r in res])
    return ksc.merge_topk(ids, dists, ip=ip)


def search_dist(shard, Q, k, nprobe, rerank, opts=None, ip=False, group=None, ops=None):
    """The sharded search with one shard per process (rank r holds shard r);
    every rank passes the same queries.  `ops` replaces the three library
    steps (candidates, rerank, merge) -- for tests of the exchanges on
    processes without a device."""
    import torch
    import torch.distributed as dist
    from . import ksc
    ws = dist.get_world_size(group)
    cand = ops["candidates"] if ops else (lambda: shard.shard_candidates(Q, k, nprobe, rerank, opts=opts))
    rer = ops["rerank"] if ops else (lambda own, allk: shard.shard_rerank(Q, k, rerank, own, allk))
    merge = ops["merge"] if ops else (lambda i, d: ksc.merge_topk(i, d, ip=ip))
    own = cand()
    gathered = [torch.empty_like(own) for _ in range(ws)]
    dist.all_gather(gathered, own, group=group)
    ids, dists = rer(own, torch.stack(gathered))
    gi = [torch.empty_like(ids) for _ in range(ws)]
    gd = [torch.empty_like(dists) for _ in range(ws)]
    dist.all_gather(gi, ids, group=group)
    dist.all_gather(gd, dists, group=group)
    return merge(torch.stack(gi), torch.stack(gd))
