"""Predictive cluster pruning (Sec. 4.2.3, Table 4, Alg. 2) on the GPU vs the
CPU oracle, through the C ABI (needs a GB300).

Per-list statistics: FP32 distances against FP64, so moments within 1e-5
relative, histogram / outlier fractions within one member, principal
variances within 1e-3 and axes within 2e-3 (both sides run the same power
iterations from the same start).  Features: the oracle is fed the GPU's own
statistics, so they agree to FP32 rounding.  Probabilities within 1e-5; the
kept probe lists equal wherever no probability lies within 1e-4 of theta.
Labels bit-exact.  The pruned search equals the search of the kept lists,
and its sampled results equal the oracle's scan + re-rank of those lists.
"""
import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

from test_gpu_parity import small_index, gpu_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    ix, Q = small_index("small")
    g = gpu_index(ksc, ix)
    g.pruner_stats()
    return torch, ksc, ix, Q, g


def _random_model(rng, feats):
    F, H = oracle.PRUNE_NFEAT, oracle.PRUNE_H
    w = rng.normal(size=oracle.mlp_nparams(F, H, H)) * 0.4
    f = feats.reshape(-1, F)
    mu, sd = f.mean(0), np.maximum(f.std(0), 1e-6)
    return np.concatenate([w, mu, sd]).astype(np.float32)


def test_stats_match_oracle(env):
    torch, ksc, ix, Q, g = env
    st_g, vec_g, _ = g.pruner_export(model=False)
    st_o, vec_o = oracle.prune_stats(ix["X"], ix["c_mean"], ix["assign"])
    n = st_o[:, 0]
    np.testing.assert_array_equal(st_g[:, 0], n)
    np.testing.assert_allclose(st_g[:, 1:4], st_o[:, 1:4], rtol=1e-5)
    one = 1.0 / np.maximum(n, 1)[:, None] + 1e-6
    assert np.all(np.abs(st_g[:, 4:9] - st_o[:, 4:9]) <= one)
    np.testing.assert_allclose(st_g[:, 9:11], st_o[:, 9:11], rtol=1e-3)
    np.testing.assert_allclose(vec_g[:, :2], vec_o[:, :2], atol=2e-3)
    same_out = np.abs(st_g[:, 8] - st_o[:, 8]) < 1e-9
    np.testing.assert_allclose(vec_g[same_out, 2], vec_o[same_out, 2], rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("per_query", [False, True])
def test_features_match_oracle(env, per_query):
    torch, ksc, ix, Q, g = env
    P = 16
    Qd = torch.from_numpy(Q).cuda()
    probes = g.rank_lists(Qd, P, want_scores=False)[0]
    npb = None
    if per_query:
        npb = torch.from_numpy(np.random.default_rng(3).integers(1, P + 1, size=len(Q)).astype(np.int32)).cuda()
    fg = g.prune_probes(Qd, probes, P=P, nprobe=npb, feats=True, kept=False)["feats"].cpu().numpy()
    st, vec, _ = g.pruner_export(model=False)
    fo = oracle.prune_features(Q, ix["c_mean"], probes.cpu().numpy(), st.astype(np.float64),
                               vec.astype(np.float64), P=P, nprobe=None if npb is None else npb.cpu().numpy())
    np.testing.assert_allclose(fg, fo, rtol=2e-4, atol=2e-5)
    if per_query:
        n = npb.cpu().numpy()
        for q in range(len(Q)):
            assert not fg[q, n[q]:].any()


def test_probabilities_and_kept_lists_match_oracle(env):
    torch, ksc, ix, Q, g = env
    P, theta = 12, 0.5
    Qd = torch.from_numpy(Q).cuda()
    probes = g.rank_lists(Qd, P, want_scores=False)[0]
    st, vec, _ = g.pruner_export(model=False)
    pn = probes.cpu().numpy()
    fo = oracle.prune_features(Q, ix["c_mean"], pn, st.astype(np.float64), vec.astype(np.float64), P=P)
    model = _random_model(np.random.default_rng(7), fo)
    g.pruner_model(set_to=model)
    np.testing.assert_array_equal(g.pruner_model(), model)
    out = g.prune_probes(Qd, probes, P=P, theta=theta, prob=True)
    NP = oracle.mlp_nparams(oracle.PRUNE_NFEAT, oracle.PRUNE_H, oracle.PRUNE_H)
    po = oracle.prune_prob(fo, model[NP:NP + 16].astype(np.float64), model[NP + 16:].astype(np.float64),
                           model[:NP].astype(np.float64))
    pg = out["prob"].cpu().numpy()
    np.testing.assert_allclose(pg, po, atol=1e-5)
    keep_o = oracle.prune_keep(po, theta, P=P)
    kp, kn = out["probes"].cpu().numpy(), out["nprobe"].cpu().numpy()
    compared = 0
    for q in range(len(Q)):
        assert kn[q] >= 1 and kp[q, 0] == pn[q, 0] and np.all(kp[q, kn[q]:] == -1)
        if np.any(np.abs(po[q, 1:P] - theta) < 1e-4):
            continue
        compared += 1
        np.testing.assert_array_equal(kp[q, :kn[q]], pn[q, keep_o[q]])
    assert compared >= len(Q) - 2
    # theta above every probability keeps rank 0 only; below, every rank
    for th, want in ((1.5, 1), (-0.5, P)):
        o = g.prune_probes(Qd, probes, P=P, theta=th)
        assert np.all(o["nprobe"].cpu().numpy() == want)


def test_labels_match_oracle(env):
    torch, ksc, ix, Q, g = env
    P, k, R = 10, 10, 100
    Qd = torch.from_numpy(Q).cuda()
    probes = g.rank_lists(Qd, P, want_scores=False)[0]
    ids, dists = g.search(Qd, k, P, R)
    _, true_d = oracle.exact_knn(Q, ix["X"], k)
    kth = true_d[:, k - 1].astype(np.float32)
    lab = g.prune_labels(ids, dists, torch.from_numpy(kth).cuda(), probes, P).cpu().numpy()
    ref = oracle.prune_labels(ids.cpu().numpy(), dists.cpu().numpy(), kth, ix["assign"], probes.cpu().numpy(), P)
    np.testing.assert_array_equal(lab, ref)
    assert lab[:, 0].mean() > 0.5 and 0 < lab.mean() < 1


def test_pruning_network_gradient_matches_oracle(env):
    torch, ksc, ix, Q, g = env
    rng = np.random.default_rng(8)
    F, H = oracle.PRUNE_NFEAT, oracle.PRUNE_H
    NP = oracle.mlp_nparams(F, H, H)
    w = (rng.normal(size=NP) * 0.3).astype(np.float32)
    x = rng.normal(size=(300, F)).astype(np.float32)
    y = (rng.uniform(size=(300, 2)) < 0.4).astype(np.float32)
    loss, grad = ksc.prune_mlp_grad(torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda(),
                                    torch.from_numpy(y).cuda())
    lo, go = oracle.mlp_grad(w.astype(np.float64), F, H, H, x, y)
    assert loss.item() == pytest.approx(lo, rel=1e-4)
    np.testing.assert_allclose(grad.cpu().numpy(), go, rtol=1e-3, atol=1e-6)


def test_pruned_search_is_the_search_of_the_kept_lists(env):
    torch, ksc, ix, Q, g = env
    P, k, R, theta = 12, 10, 100, 0.5
    Qd = torch.from_numpy(Q).cuda()
    probes = g.rank_lists(Qd, P, want_scores=False)[0]
    st, vec, _ = g.pruner_export(model=False)
    fo = oracle.prune_features(Q, ix["c_mean"], probes.cpu().numpy(), st.astype(np.float64),
                               vec.astype(np.float64), P=P)
    g.pruner_model(set_to=_random_model(np.random.default_rng(9), fo))
    ids, dists, npb = g.search_pruned(Qd, k, P, R, theta)
    kept = g.prune_probes(Qd, probes, P=P, theta=theta)
    np.testing.assert_array_equal(npb.cpu().numpy(), kept["nprobe"].cpu().numpy())
    assert 1 <= npb.float().mean().item() < P
    i2, d2 = g.search_with_probes(Qd, kept["probes"], k, R)[:2]
    assert torch.equal(ids, i2) and torch.equal(dists, d2)
    kp, kn = kept["probes"].cpu().numpy(), kept["nprobe"].cpu().numpy()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    for qi in np.random.default_rng(10).choice(len(Q), 12, replace=False):
        p = kp[qi, :kn[qi]]
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, p)
        cand = oracle.scan_topr(ix, p, Ql, b, R)
        ref_ids, ref_d = oracle.rerank(Q[qi], ix, oracle.key_id(cand).astype(np.int32), k)
        np.testing.assert_allclose(dists[qi], ref_d, rtol=1e-4, atol=1e-4)
        same = ids[qi] == ref_ids
        assert same.mean() >= 0.8  # the rest tie within the tolerance above


def test_trained_pruner_drops_lists_and_keeps_recall(env):
    torch, ksc, ix, Q, g = env
    P, k, R = 16, 10, 100
    T = synth.queries(1, 3000, stream=7)
    _, tdist = oracle.exact_knn(T, ix["X"], k)
    kth = torch.from_numpy(tdist[:, k - 1].astype(np.float32)).cuda()
    Td = torch.from_numpy(T).cuda()
    loss = g.train_pruner(Td, kth, k=k, P=P, R=R, epochs=6, batch=512)
    # the loss sums the two heads' cross-entropy; a constant predictor at the
    # label rate r scores 2 H(r)
    tp = g.rank_lists(Td, P, want_scores=False)[0]
    ti, tdd = g.search_with_probes(Td, tp, k, R)[:2]
    r = g.prune_labels(ti, tdd, kth, tp, P).mean().item()
    h = -(r * np.log(r) + (1 - r) * np.log(1 - r))
    assert 0.0 < loss < 0.8 * 2 * h, (loss, r)
    Qd = torch.from_numpy(Q).cuda()
    _, true_d = oracle.exact_knn(Q, ix["X"], k)
    ids, _ = g.search(Qd, k, P, R)
    rec_full = oracle.recall(Q, ix["X"], ids.cpu().numpy(), true_d, k)
    ids, _, npb = g.search_pruned(Qd, k, P, R, 0.1)
    rec = oracle.recall(Q, ix["X"], ids.cpu().numpy(), true_d, k)
    mean_p = npb.float().mean().item()
    print("pruned: mean lists %.2f of %d, recall %.4f (unpruned %.4f), loss %.4f" % (mean_p, P, rec, rec_full, loss))
    assert mean_p < 0.8 * P
    assert rec >= rec_full - 0.03


def test_adaptive_search_prunes_its_predicted_lists(env):
    torch, ksc, ix, Q, g = env
    k, R = 10, 100
    T = synth.queries(1, 2000, stream=8)
    _, tdist = oracle.exact_knn(T, ix["X"], k)
    Td = torch.from_numpy(T).cuda()
    kth = torch.from_numpy(tdist[:, k - 1].astype(np.float32)).cuda()
    g.train_predictor(Td, kth, k=k, epochs=2)
    g.train_pruner(Td, kth, k=k, P=16, R=R, epochs=2, batch=512)
    # fixed rerank depth, so the pruned lists alone decide the result
    g.set_predictor_params(2, 16, R, R, 0.2, 0.5, 0.0, 0.0)
    Qd = torch.from_numpy(Q).cuda()
    g.pruner_theta(-1.0)
    _, _, npred, _ = g.search_adaptive(Qd, k)
    theta = 0.3
    g.pruner_theta(theta)
    ids, dists, nsearch, _ = g.search_adaptive(Qd, k)
    probes = g.rank_lists(Qd, 16, want_scores=False)[0]
    kept = g.prune_probes(Qd, probes, nprobe=npred, theta=theta)
    np.testing.assert_array_equal(nsearch.cpu().numpy(), kept["nprobe"].cpu().numpy())
    assert np.all(nsearch.cpu().numpy() <= npred.cpu().numpy())
    i2, d2 = g.search_with_probes(Qd, kept["probes"], k, R)[:2]
    assert torch.equal(ids, i2) and torch.equal(dists, d2)
    # a captured adaptive plan (capture needs a stream of its own) follows
    # the threshold too, re-capturing after it changes
    torch.cuda.synchronize()
    s_ = torch.cuda.Stream()
    with torch.cuda.stream(s_):
        pl = g.plan(len(Q), k, adaptive=True)
        i3, d3 = [t.clone() for t in pl.execute(Qd)]
        g.pruner_theta(-1.0)
        i4, d4 = [t.clone() for t in pl.execute(Qd)]
    s_.synchronize()
    assert torch.equal(i3, ids) and torch.equal(d3, dists)
    i5, d5, _, _ = g.search_adaptive(Qd, k)
    assert torch.equal(i4, i5) and torch.equal(d4, d5)
