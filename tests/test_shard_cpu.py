"""Host side of the list-sharded search on CPU (gloo, world size 2).

paper_2511_03298_gb300.shard.search_dist runs the protocol's two exchanges
(every shard's candidate keys, then every shard's (distance, id) results)
with torch.distributed all-gathers.  Here two spawned processes each hold one
shard of the same oracle-built index and replace the three library steps by
the oracle on their own lists: the exchanges must deliver the keys and results
in shard order so that the merged result equals the oracle's unsharded search.
"""
import os
import socket

import numpy as np

import pytest

KEY_NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _index():
    import oracle
    rng = np.random.default_rng(21)
    centres = rng.uniform(-4, 4, size=(10, 24))
    X = (centres[rng.integers(0, 10, 3000)] + rng.normal(size=(3000, 24))).astype(np.float32)
    Q = (centres[rng.integers(0, 10, 12)] + rng.normal(size=(12, 24))).astype(np.float32)
    ix = oracle.build_index(X, 16, 12, False, rng.permutation(3000).astype(np.int64), iters=5)
    return ix, Q


def _worker(rank, ws, port, nprobe, R, k, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2511_03298_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ix, Q = _index()
    sizes = np.diff(ix["list_off"])
    owner = shard.owners_round_robin(sizes, ws)
    probes = [oracle.rank(q, ix["c_rank"], False, nprobe)[0] for q in Q]

    def candidates():
        keys = np.full((len(Q), R), KEY_NONE, np.uint64)
        for qi, q in enumerate(Q):
            Ql, b, _ = oracle.lut_q8(q, ix, probes[qi])  # tables of the whole probe set
            mine = np.flatnonzero(owner[probes[qi]] == rank)
            if len(mine):
                kk = oracle.scan_topr(ix, probes[qi][mine], Ql[mine], b[mine], R)
                keys[qi, :len(kk)] = kk
        return torch.from_numpy(keys.view(np.int64))

    def rerank(own, allk):
        own = own.numpy().view(np.uint64)
        allk = allk.numpy().view(np.uint64)  # [parts x nq x R]
        ids = np.full((len(Q), k), -1, np.int64)
        dd = np.full((len(Q), k), np.inf)
        for qi, q in enumerate(Q):
            theta = np.sort(allk[:, qi, :].ravel())[R - 1]
            mine = own[qi][(own[qi] != KEY_NONE) & (own[qi] <= theta)]
            if len(mine):
                i_, d_ = oracle.rerank(q, ix, oracle.key_id(mine).astype(np.int32), k)
                ids[qi], dd[qi] = i_, d_
        return torch.from_numpy(ids), torch.from_numpy(dd)

    def merge(gi, gd):
        gi, gd = gi.numpy(), gd.numpy()  # [parts x nq x k]
        ids = np.zeros((len(Q), k), np.int64)
        dd = np.zeros((len(Q), k))
        for qi in range(len(Q)):
            i_, d_ = gi[:, qi, :].ravel(), gd[:, qi, :].ravel()
            idk = np.where(i_ < 0, np.iinfo(np.int64).max, i_)
            o = np.lexsort((idk, d_))[:k]
            ids[qi], dd[qi] = i_[o], d_[o]
        return ids, dd

    ids, dd = shard.search_dist(None, None, k, nprobe, R,
                                ops={"candidates": candidates, "rerank": rerank, "merge": merge})
    dist.destroy_process_group()
    out.put(dict(rank=rank, ids=ids.tolist(), d=dd.tolist()))


def test_two_shards_exchange_and_merge_to_the_unsharded_result():
    import torch.multiprocessing as mp
    import oracle
    ws, nprobe, R, k = 2, 6, 60, 10
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, ws, port, nprobe, R, k, out)) for r in range(ws)]
    for p in ps:
        p.start()
    try:
        res = [out.get(timeout=240) for _ in range(ws)]
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
    ix, Q = _index()
    ref = oracle.search(ix, Q, nprobe, R, k)
    for r_ in res:
        assert np.array_equal(np.array(r_["ids"]), ref["ids"])
        np.testing.assert_array_equal(np.array(r_["d"]), ref["dists"])


def test_round_robin_owners_balance_vectors():
    from paper_2511_03298_gb300 import shard
    sizes = np.array([50, 10, 40, 30, 20, 0, 5])
    own = shard.owners_round_robin(sizes, 3)
    loads = np.bincount(own, weights=sizes, minlength=3)
    assert sorted(loads.tolist()) == [50.0, 50.0, 55.0]
    assert np.array_equal(shard.owners_round_robin(sizes, 1), np.zeros(7, np.int32))
