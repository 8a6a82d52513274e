"""List-sharded search on one GPU: G shards of one index (each a separate
index object holding only its lists' vectors) give the unsharded search's
results bit for bit, through the library's three steps and the exchanges of
paper_2511_03298_gb300.shard.search_local."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc, shard
    return torch, ksc, shard


def _index(kind):
    rng = np.random.default_rng(31 if kind == "l2" else 32)
    d = 64 if kind == "l2" else 48
    centres = rng.uniform(-4, 4, size=(16, d))
    X = (centres[rng.integers(0, 16, 8000)] + rng.normal(size=(8000, d))).astype(np.float32)
    Q = (centres[rng.integers(0, 16, 64)] + rng.normal(size=(64, d))).astype(np.float32)
    ip = kind == "ip"
    if ip:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    ix = oracle.build_index(X, 40, d // 2, ip, rng.permutation(8000).astype(np.int64), iters=5, ip=ip)
    return ix, Q


@pytest.mark.parametrize("kind", ["l2", "ip"])
@pytest.mark.parametrize("G", [2, 3])
@pytest.mark.parametrize("nq", [64, 1600])
def test_sharded_search_equals_unsharded(env, kind, G, nq):
    torch, ksc, shard = env
    ix, Q = _index(kind)
    metric = "ip" if kind == "ip" else "l2"
    full = ksc.index_import(ix, metric=metric, spherical=ix["spherical"])
    sizes = np.diff(ix["list_off"])
    owner = shard.owners_round_robin(sizes, G)
    shards = [ksc.index_import_shard(ix, owner, g, metric=metric, spherical=ix["spherical"]) for g in range(G)]
    assert sum(s.info()["n"] for s in shards) == ix["n"]
    Qd = torch.from_numpy(np.tile(Q, (nq // len(Q), 1))).cuda()
    k, P, R = 10, 7, 120
    ref = full.search(Qd, k, P, R)
    got = shard.search_local(shards, Qd, k, P, R, ip=kind == "ip")
    assert torch.equal(got[0], ref[0])
    assert torch.equal(got[1], ref[1])
    # the shards' keys at or below the whole index's R-th key are exactly the
    # unsharded candidates (same probes through the whole index's ranking)
    probes, _ = full.rank_lists(Qd[:16], P)
    _, _, cand, ncand = full.search_with_probes(Qd[:16], probes, k, R)
    own = [s.shard_candidates(Qd[:16], k, P, R).cpu().numpy().view(np.uint64) for s in shards]
    cand = cand.cpu().numpy().view(np.uint64)
    for qi in range(16):
        allk = np.sort(np.concatenate([o[qi] for o in own]))
        assert np.array_equal(allk[:ncand[qi].item()], cand[qi, :ncand[qi].item()])
    for s in shards:
        assert s.last_status() == 0


def test_skewed_partition_and_unprobed_shard(env):
    """One shard owns a single list that few queries probe: its candidate
    lists are mostly padding, and the merge still gives the unsharded
    result."""
    torch, ksc, shard = env
    ix, Q = _index("l2")
    full = ksc.index_import(ix)
    sizes = np.diff(ix["list_off"])
    nonempty = np.flatnonzero(sizes > 0)
    owner = np.zeros(ix["L"], np.int32)
    owner[int(nonempty[np.argmin(sizes[nonempty])])] = 1
    shards = [ksc.index_import_shard(ix, owner, g) for g in range(2)]
    Qd = torch.from_numpy(Q).cuda()
    ref = full.search(Qd, 10, 5, 100)
    got = shard.search_local(shards, Qd, 10, 5, 100)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_shard_argument_errors(env):
    torch, ksc, shard = env
    ix, Q = _index("l2")
    owner = np.zeros(ix["L"], np.int32)
    with pytest.raises(ksc.KscError, match="holds no vector"):
        ksc.index_import_shard(ix, owner, 1)
    full = ksc.index_import(ix)
    with pytest.raises(ksc.KscError, match="not a shard"):
        full.shard_candidates(torch.from_numpy(Q).cuda(), 10, 4, 100)
