"""Handles on the same index data with their own workspaces (ksc_index_view):
searches through them on different streams at the same time give the same
results as the same searches one after another (needs a GB300)."""
import numpy as np
import pytest

from paper_2511_03298_gb300 import synth

from test_gpu_parity import small_index, gpu_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    ix, _ = small_index("small")
    return torch, ksc, gpu_index(ksc, ix)


def test_concurrent_searches_through_views(env):
    torch, ksc, g = env
    k, P, R = 10, 8, 100
    batches = [torch.from_numpy(synth.queries(1, n, stream=s)).cuda() for s, n in ((11, 700), (12, 1), (13, 257))]
    ref = [g.search(Q, k, P, R) for Q in batches]
    torch.cuda.synchronize()
    views = [g, g.view(), g.view()]
    streams = [torch.cuda.Stream() for _ in views]
    outs = []
    for rep in range(3):
        res = [None] * 3
        for i, (v, s_) in enumerate(zip(views, streams)):
            with torch.cuda.stream(s_):
                res[i] = v.search(batches[i], k, P, R)
        torch.cuda.synchronize()
        outs.append(res)
    for res in outs:
        for (i1, d1), (i2, d2) in zip(res, ref):
            assert torch.equal(i1, i2) and torch.equal(d1, d2)
    # a captured plan per view, replayed on its own stream
    plans = []
    for v, s_, Q in zip(views, streams, batches):
        with torch.cuda.stream(s_):
            plans.append(v.plan(Q.shape[0], k, nprobe=P, rerank=R))
    got = [None] * 3
    for i, (pl, s_, Q) in enumerate(zip(plans, streams, batches)):
        with torch.cuda.stream(s_):
            got[i] = [t.clone() for t in pl.execute(Q)]
    torch.cuda.synchronize()
    for (i1, d1), (i2, d2) in zip(got, ref):
        assert torch.equal(i1, i2) and torch.equal(d1, d2)
    del plans, got


def test_views_do_not_train_and_free_first(env):
    torch, ksc, g = env
    v = g.view()
    T = torch.from_numpy(synth.queries(1, 64, stream=14)).cuda()
    kth = torch.ones(64, dtype=torch.float32, device="cuda")
    with pytest.raises(ksc.KscError):
        v.train_pruner(T, kth)
    with pytest.raises(ksc.KscError):
        v.pruner_stats()
    ids_v, _ = v.search(T, 10, 8, 100)
    v.free()
    ids_g, _ = g.search(T, 10, 8, 100)
    assert torch.equal(ids_v, ids_g)
