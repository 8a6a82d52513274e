"""Full-size sampled parity for the two larger workloads (needs a GB300).

- 10M x 96 unit-norm vectors, nlist 8192, M 48, k 100, rerank 1000, per-query
  nprobe U{4..256} (the batched configuration): results of sampled queries
  equal the oracle's scan + FP32 re-rank on the same index and probes, and a
  query's result does not depend on the batch it is searched in.
- 1.2M x 100 unit-norm vectors, inner product, nlist 2048, M 50 (d' = 2):
  candidates of sampled queries bit-exact; the BF16 / FP8 first re-rank keeps
  a shortlist of the candidates whose FP32 re-rank the oracle reproduces.
"""
import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    return torch, ksc


def _same_results(ix, q, ids, dists, ref_ids, ref_d):
    """Top-k equal up to exact-distance ties within RTOL."""
    np.testing.assert_allclose(dists, ref_d, rtol=RTOL, atol=1e-4)
    X = ix["X"]
    for r in range(len(ids)):
        if ids[r] == ref_ids[r]:
            continue
        assert ids[r] >= 0 and ref_ids[r] >= 0
        x = X[ids[r]].astype(np.float64)
        qd = q.astype(np.float64)
        exact = (qd @ x) if ix["ip"] else ((qd - x) ** 2).sum()  # IP results carry q.x
        assert abs(exact - ref_d[r]) <= RTOL * max(1.0, abs(ref_d[r])), (r, exact, ref_d[r])


def test_full_size_deep_sampled_parity(env):
    torch, ksc = env
    c = synth.CONFIGS[4]
    X = synth.base(4)
    nq, k, R, Pmax = 4096, c["k"], c["R"], 256
    Q = synth.queries(4, nq)
    npb = synth.per_query_nprobe(4, nq)
    g = ksc.build_index(torch.from_numpy(X).cuda(), c["L"], c["M"], spherical=True,
                        perm=synth.build_perm(4, len(X)))
    Qd = torch.from_numpy(Q).cuda()
    npb_d = torch.from_numpy(npb).cuda()
    rr = torch.full((nq,), R, dtype=torch.int32, device="cuda")
    ids, dists = g.search_varprobe(Qd, k, npb_d, rr, nprobe_max=Pmax, rerank_max=R)
    probes = g.rank_lists(Qd, Pmax, want_scores=False)[0].cpu().numpy()
    # batch independence: sub-batches of 1, 16 and 256 queries give the same rows
    for B in (1, 16, 256):
        i2, d2 = g.search_varprobe(Qd[:B], k, npb_d[:B], rr[:B], nprobe_max=Pmax, rerank_max=R)
        assert torch.equal(i2, ids[:B]) and torch.equal(d2, dists[:B]), B
    e = g.export()
    ix = oracle.make_index(X, e["c_rank"], e["c_mean"], e["codebook"], e["codes"], e["assign"], spherical=True)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    sample = np.random.default_rng(11).choice(nq, 12, replace=False)
    for qi in sample:
        p = probes[qi, :npb[qi]]
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, p)
        cand = oracle.scan_topr(ix, p, Ql, b, R)
        ref_ids, ref_d = oracle.rerank(Q[qi], ix, oracle.key_id(cand).astype(np.int32), k)
        _same_results(ix, Q[qi], ids[qi], dists[qi], ref_ids, ref_d)


def test_full_size_glove_sampled_parity(env):
    torch, ksc = env
    c = synth.CONFIGS[3]
    X = synth.base(3)
    Q = synth.queries(3)
    g = ksc.build_index(torch.from_numpy(X).cuda(), c["L"], c["M"], metric="ip", spherical=True,
                        perm=synth.build_perm(3, len(X)))
    e = g.export()
    ix = oracle.make_index(X, e["c_rank"], e["c_mean"], e["codebook"], e["codes"], e["assign"], ip=True,
                           spherical=True)
    P, Rw, Rf, k = 32, 800, 100, c["k"]
    Qd = torch.from_numpy(Q).cuda()
    gp = g.rank_lists(Qd, P, want_scores=False)[0]
    out = {}
    for prec in (0, 1, 2):
        opts = None if prec == 0 else ksc.search_opts(precision=prec, rerank_final=Rf)
        out[prec] = [t.cpu().numpy() for t in g.search_with_probes(Qd, gp, k, Rw, opts=opts)]
    gp = gp.cpu().numpy()
    for prec in (1, 2):  # the scan does not depend on the re-rank precision
        assert np.array_equal(out[prec][2], out[0][2]) and np.array_equal(out[prec][3], out[0][3])
    sample = np.random.default_rng(13).choice(len(Q), 30, replace=False)
    overlap = {1: [], 2: []}
    for qi in sample:
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, gp[qi])
        cand = oracle.scan_topr(ix, gp[qi], Ql, b, Rw)
        assert np.array_equal(out[0][2][qi].view(np.uint64), cand), qi
        cid = oracle.key_id(cand).astype(np.int32)
        ref_ids, ref_d = oracle.rerank(Q[qi], ix, cid, k)
        _same_results(ix, Q[qi], out[0][0][qi], out[0][1][qi], ref_ids, ref_d)
        for prec in (1, 2):
            ids, dists = out[prec][0][qi], out[prec][1][qi]
            assert np.all(np.isin(ids, cid)), (prec, qi)
            # the final stage is the FP32 re-rank of the shortlist
            s_ids, s_d = oracle.rerank(Q[qi], ix, ids.astype(np.int32), k)
            _same_results(ix, Q[qi], ids, dists, s_ids, s_d)
            overlap[prec].append(len(np.intersect1d(ids, ref_ids)) / k)
    for prec in (1, 2):
        print("precision %d: mean top-%d overlap with the FP32 re-rank of all %d = %.3f"
              % (prec, k, Rw, np.mean(overlap[prec])))
        assert np.mean(overlap[prec]) >= 0.9, prec
