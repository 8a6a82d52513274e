"""Component filtration (Sec. 4.3, Alg. 1 / Alg. 2) on the GPU vs the CPU
oracle, through the C ABI (needs a GB300).

Column statistics: means and standard deviations within 1e-12 relative of the
oracle's FP64 (same arithmetic, another summation order), fractions equal
(integer counts; a value exactly on the one-std boundary could move one).
The filtered index keeps the oracle's dimensions; with given probes its
candidates equal the oracle's scan of the filtered vectors bit for bit, and
its distances the oracle's re-rank with the full query against the full
vectors (1e-4 relative).
"""
import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

pytestmark = pytest.mark.gpu

THR = 0.99
N = 6000


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    X = synth.base(6, n=N)
    Q = synth.queries(6, 60)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 32, 196, filter_threshold=THR, iters=10,
                        perm=synth.build_perm(6, N))
    return torch, ksc, X, Q, g


def test_component_stats_match_oracle(env):
    torch, ksc, X, Q, g = env
    rng = np.random.default_rng(1)
    Y = np.concatenate([X[:, :200], rng.normal(size=(N, 7)).astype(np.float32), np.zeros((N, 1), np.float32)], 1)
    mu, sd, fr = [t.cpu().numpy() for t in ksc.component_stats(torch.from_numpy(np.ascontiguousarray(Y)).cuda())]
    mo, so, fo = oracle.component_stats(Y)
    np.testing.assert_allclose(mu, mo, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sd, so, rtol=1e-12, atol=1e-12)
    assert np.all(np.abs(fr - fo) <= 1.0 / N + 1e-15)


def test_filtered_index_keeps_the_oracle_dimensions(env):
    torch, ksc, X, Q, g = env
    dfull, dims = g.dims()
    _, _, fo = oracle.component_stats(X)
    want = oracle.component_dims(oracle.component_keep(fo, THR), 144)
    assert dfull == 784
    np.testing.assert_array_equal(dims, want)
    inf = g.info()
    assert inf["d"] == len(want) and inf["M"] == len(want) // 4  # sub-vector width d / M = 4 kept


def test_filtered_search_matches_oracle(env):
    torch, ksc, X, Q, g = env
    P, k, R = 6, 10, 50
    _, dims = g.dims()
    e = g.export()
    ix = oracle.make_index(e["X"], e["c_rank"], e["c_mean"], e["codebook"], e["codes"], e["assign"])
    np.testing.assert_array_equal(e["X"], oracle.filter_rows(X, dims))
    Qw = oracle.filter_rows(Q, dims)
    probes = np.stack([oracle.rank(q, ix["c_rank"], False, P)[0] for q in Qw]).astype(np.int32)
    Qd = torch.from_numpy(Q).cuda()
    ids, dists, cand, ncand = g.search_with_probes(Qd, torch.from_numpy(probes).cuda(), k, R)
    ids, dists, cand = ids.cpu().numpy(), dists.cpu().numpy(), cand.cpu().numpy()
    full = dict(X=X, d=X.shape[1], ip=False)
    for qi in range(len(Q)):
        Ql, b, _ = oracle.lut_q8(Qw[qi], ix, probes[qi])
        ref = oracle.scan_topr(ix, probes[qi], Ql, b, R)
        np.testing.assert_array_equal(cand[qi].view(np.uint64), ref)
        ref_ids, ref_d = oracle.rerank(Q[qi], full, oracle.key_id(ref).astype(np.int32), k)
        np.testing.assert_allclose(dists[qi], ref_d, rtol=1e-4, atol=1e-3)
        assert (ids[qi] == ref_ids).mean() >= 0.8  # the rest tie within the tolerance above


def test_filtered_search_entry_points_agree(env):
    torch, ksc, X, Q, g = env
    P, k, R = 8, 10, 50
    Qd = torch.from_numpy(Q).cuda()
    ids, dists = g.search(Qd, k, P, R)
    probes = g.rank_lists(Qd, P, want_scores=False)[0]
    i2, d2 = g.search_with_probes(Qd, probes, k, R)[:2]
    assert torch.equal(ids, i2) and torch.equal(dists, d2)
    npb = torch.full((len(Q),), P, dtype=torch.int32, device="cuda")
    rr = torch.full((len(Q),), R, dtype=torch.int32, device="cuda")
    i3, d3 = g.search_varprobe(Qd, k, npb, rr, nprobe_max=P, rerank_max=R)
    assert torch.equal(ids, i3) and torch.equal(dists, d3)
    torch.cuda.synchronize()
    s_ = torch.cuda.Stream()
    with torch.cuda.stream(s_):
        pl = g.plan(len(Q), k, nprobe=P, rerank=R)
        i4, d4 = [t.clone() for t in pl.execute(Qd)]
    s_.synchronize()
    assert torch.equal(ids, i4) and torch.equal(dists, d4)
    # the re-rank distances are those of the full vectors
    full = ((Q[:, None, :].astype(np.float64) - X[ids.cpu().numpy()].astype(np.float64)) ** 2).sum(-1)
    np.testing.assert_allclose(dists.cpu().numpy(), full, rtol=1e-4, atol=1e-2)
    # recall close to an unfiltered index of the same data
    _, true_d = oracle.exact_knn(Q, X, k)
    u = ksc.build_index(torch.from_numpy(X).cuda(), 32, 196, iters=10, perm=synth.build_perm(6, N))
    iu, _ = u.search(Qd, k, P, R)
    rf = oracle.recall(Q, X, ids.cpu().numpy(), true_d, k)
    ru = oracle.recall(Q, X, iu.cpu().numpy(), true_d, k)
    print("recall@10 filtered %.4f unfiltered %.4f" % (rf, ru))
    assert rf >= ru - 0.05
