"""Batched execution: CUDA-graph plans and the autotuner.

A captured plan must return exactly what the direct search returns, also
after another search has reallocated the index workspace (the plan then
re-captures).  Every configuration the autotuner tries is an exact variant
(same candidates), so its choice must leave results unchanged.
"""
import numpy as np
import pytest

from paper_2511_03298_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    X = synth.base(2, n=100_000)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 256, 64, perm=synth.build_perm(2, len(X)), iters=8)
    return torch, ksc, g


def test_plan_replay_equals_direct_search(env):
    torch, ksc, g = env
    st = torch.cuda.Stream()
    Q1 = torch.from_numpy(synth.queries(2, 300)).cuda()
    Q2 = torch.from_numpy(synth.rng_array(7, (300, 128), "uniform") * 255).cuda()
    with torch.cuda.stream(st):
        ref1 = g.search(Q1, 10, 8, 200)
        ref2 = g.search(Q2, 10, 8, 200)
        plan = g.plan(300, 10, nprobe=8, rerank=200)
        a = plan.execute(Q1)
        b = plan.execute(Q2)
        # a larger search grows the workspace; the plan must re-capture
        big = torch.from_numpy(synth.queries(2, 3000)).cuda()
        g.search(big, 10, 32, 400)
        c = plan.execute(Q1)
    st.synchronize()
    for (x, y) in ((a, ref1), (b, ref2), (c, ref1)):
        assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])


def test_plan_of_the_adaptive_search(env):
    torch, ksc, g = env
    rng = np.random.default_rng(3)
    g.predictor_weights(set_to=rng.normal(scale=0.1, size=8450))
    g.set_predictor_params(pmin=2, pmax=16, rmin=50, rmax=200, p0=0.2, p1=0.5, r0=0.2, r1=0.5)
    st = torch.cuda.Stream()
    Q = torch.from_numpy(synth.queries(2, 200)).cuda()
    with torch.cuda.stream(st):
        ref = g.search_adaptive(Q, 10)
        plan = g.plan(200, 10, adaptive=True)
        got = plan.execute(Q)
    st.synchronize()
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_autotune_picks_an_exact_configuration(env):
    torch, ksc, g = env
    Q = torch.from_numpy(synth.queries(2, 1000)).cuda()
    opts, ms = g.autotune(Q, 10, 12, 200)
    assert opts.lanes_per_query in (4, 8, 16, 32) and opts.tile_blocks in (0, 8, 16, 32, 64) and ms > 0
    a = g.search(Q, 10, 12, 200)
    b = g.search(Q, 10, 12, 200, opts=opts)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
