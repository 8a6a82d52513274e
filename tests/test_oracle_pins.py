"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine that computes the same textbook quantity, a closed form, an exact
rational computation, brute force on tiny inputs, or an invariant.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2511_03298_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_index(orc, n=3000, d=16, L=8, M=8, seed=0, ip=False):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-4, 4, size=(L, d))
    X = (centres[rng.integers(0, L, n)] + rng.normal(size=(n, d))).astype(np.float32)
    if ip:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
    perm = rng.permutation(n).astype(np.int64)
    return orc.build_index(X, L, M, spherical=ip, perm=perm, iters=10, ip=ip), rng


# ---------------------------------------------------------------- k-means
def test_kmeans_matches_scipy_lloyd(orc):
    """Lloyd iterations (Sec. 2.2) equal scipy's kmeans2 from the same init on
    separated data (no ties, no empty clusters)."""
    from scipy.cluster.vq import kmeans2
    rng = np.random.default_rng(1)
    centres = rng.uniform(-20, 20, size=(6, 5))
    X = (centres[rng.integers(0, 6, 2000)] + rng.normal(size=(2000, 5))).astype(np.float32)
    sample = np.arange(2000, dtype=np.int64)
    for iters in (1, 3, 10):
        Cc, _ = orc.kmeans(X, sample, 6, iters)
        ref, _ = kmeans2(X.astype(np.float64), X[:6].astype(np.float64), iter=iters, minit="matrix")
        np.testing.assert_allclose(Cc, ref, rtol=1e-10, atol=1e-10)


def test_kmeans_objective_non_increasing_and_single_cluster_mean(orc):
    X = synth.base(1, n=4000)
    sample = synth.build_perm(1, 4000)[:2000]
    _, obj = orc.kmeans(X, sample, 16, 8)
    assert np.all(np.diff(obj) <= 1e-9 * obj[0])
    # L = 1: the single centroid is the mean of the sample (closed form)
    Cc, obj1 = orc.kmeans(X, sample, 1, 2)
    np.testing.assert_allclose(Cc[0], X[sample].astype(np.float64).mean(0), rtol=1e-12, atol=1e-12)
    assert np.isclose(obj1[-1], ((X[sample] - Cc[0]) ** 2).sum(), rtol=1e-9)


def test_kmeans_tie_to_lower_id_and_empty_keeps(orc):
    # two identical init points: all points tie -> lower id takes them, the
    # other cluster stays empty and keeps its centroid.
    X = np.array([[0, 0], [0, 0], [1, 0], [2, 0]], np.float32)
    Cc, _ = orc.kmeans(X, np.arange(4, dtype=np.int64), 2, 1)
    np.testing.assert_allclose(Cc[0], [0.75, 0.0])
    np.testing.assert_allclose(Cc[1], [0.0, 0.0])
    # second step: the duplicated origin points now go to centroid 1
    Cc, _ = orc.kmeans(X, np.arange(4, dtype=np.int64), 2, 3)
    np.testing.assert_allclose(Cc, [[1.5, 0.0], [0.0, 0.0]])


# ---------------------------------------------------------------- encode
def test_encode_separable_equals_joint_bruteforce(orc):
    """Sec. 2.3: per-subspace argmin equals the joint argmin over all 16^2
    codeword pairs of the reconstruction error (M = 2)."""
    rng = np.random.default_rng(2)
    d, M = 6, 2
    cb = rng.normal(size=(M, 16, d // M)).astype(np.float32)
    R = rng.normal(size=(200, d)).astype(np.float32)
    codes, _ = orc.encode(R, M, cb)
    for r, c in zip(R, codes):
        best, arg = np.inf, None
        for i0 in range(16):
            for i1 in range(16):
                rec = np.concatenate([cb[0, i0], cb[1, i1]]).astype(np.float64)
                e = ((r - rec) ** 2).sum()
                if e < best:
                    best, arg = e, (i0, i1)
        assert tuple(c) == arg


# ---------------------------------------------------------------- index build
@pytest.mark.parametrize("ip", [False, True])
def test_build_index_invariants(orc, ip):
    ix, _ = tiny_index(orc, ip=ip)
    X, a, L = ix["X"], ix["assign"], ix["L"]
    # assignment = lowest ranking score (scipy cdist / dot as the library routine)
    from scipy.spatial.distance import cdist
    if ip:
        s = -(X.astype(np.float64) @ ix["c_rank"].astype(np.float64).T)
        np.testing.assert_allclose(np.linalg.norm(ix["c_rank"], axis=1), 1.0, rtol=1e-6)
    else:
        s = cdist(X.astype(np.float64), ix["c_rank"].astype(np.float64), "sqeuclidean")
    assert np.array_equal(a, np.argmin(s, axis=1))
    # residual centroid = arithmetic mean of members (Sec. 4.6.1)
    for c in range(L):
        mem = X[a == c]
        if len(mem):
            np.testing.assert_allclose(ix["c_mean"][c], mem.astype(np.float64).mean(0), rtol=1e-5, atol=1e-6)
    # codes = nearest codeword of the stored fp32 residual
    Rres = X - ix["c_mean"][a]
    codes2, _ = orc.encode(Rres, ix["M"], ix["codebook"])
    assert np.array_equal(codes2, ix["codes"])


def test_mean_centroid_residual_is_tighter_than_normalised(orc):
    """Sec. 4.6.1: on unit-norm data the arithmetic-mean centroid gives a
    smaller residual energy than the normalised centroid in every cluster
    (the mean minimises the sum of squares)."""
    ix, _ = tiny_index(orc, ip=True)
    X, a = ix["X"].astype(np.float64), ix["assign"]
    for c in range(ix["L"]):
        mem = X[a == c]
        if len(mem) == 0:
            continue
        e_mean = ((mem - ix["c_mean"][c]) ** 2).sum()
        e_norm = ((mem - ix["c_rank"][c]) ** 2).sum()
        assert e_mean <= e_norm * (1 + 1e-6)


# ---------------------------------------------------------------- ranking
@pytest.mark.parametrize("spherical", [False, True])
def test_rank_matches_library_sort(orc, spherical):
    rng = np.random.default_rng(3)
    C_ = rng.normal(size=(300, 12)).astype(np.float32)
    C_[17] = C_[5]  # exact tie: lower id first
    q = rng.normal(size=12).astype(np.float32)
    probes, scores = orc.rank(q, C_, spherical, 40)
    from scipy.spatial.distance import cdist
    s = (-(C_.astype(np.float64) @ q.astype(np.float64)) if spherical
         else cdist(q[None].astype(np.float64), C_.astype(np.float64), "sqeuclidean")[0])
    order = np.lexsort((np.arange(300), s))[:40]
    assert np.array_equal(probes, order)


# ---------------------------------------------------------------- ADC (Eq. 1)
@pytest.mark.parametrize("ip", [False, True])
def test_adc_equals_reconstructed_vector_distance(orc, ip):
    """Eq. 1 with residual tables equals the distance to the reconstructed
    vector c_p + r_hat (an identity, so FP64 round-off only)."""
    ix, rng = tiny_index(orc, ip=ip)
    d, M = ix["d"], ix["M"]
    ds = d // M
    for _ in range(200):
        q = rng.normal(size=d).astype(np.float32)
        i = int(rng.integers(0, ix["n"]))
        p = int(ix["assign"][i])
        code = ix["codes"][i]
        rec = ix["c_mean"][p].astype(np.float64) + np.concatenate(
            [ix["codebook"][j, code[j]] for j in range(M)]).astype(np.float64)
        ref = -(q.astype(np.float64) @ rec) if ip else ((q - rec) ** 2).sum()
        got = orc.adc64(q, ix, p, code)
        assert abs(got - ref) <= 1e-9 * (1 + abs(ref))
        assert ds * M == d


# ---------------------------------------------------------------- quantised LUT
def test_lut_q8_worked_example_exact_rationals(orc):
    """8-bit LUT (Sec. 2.5, Sec. 4.5) on a hand example with integer tables,
    checked against exact rational arithmetic (tests/golden/lut_q8_worked.json)."""
    g = json.load(open(os.path.join(GOLDEN, "lut_q8_worked.json")))
    q = np.array(g["q"], np.float32)
    cb = np.array(g["codebook"], np.float32)
    c_mean = np.array(g["c_mean"], np.float32)
    X = np.zeros((1, len(q)), np.float32)
    ix = orc.make_index(X, c_mean, c_mean, cb, np.zeros((1, cb.shape[0]), np.uint8),
                        np.zeros(1, np.int32))
    Q, bias, a = orc.lut_q8(q, ix, np.array([0], np.int32))
    # exact: T_j[i] integers; R = max range; Q = floor((T - m) * 255/R + 1/2)
    T = [[sum((Fraction(float(q[j * 2 + t])) - Fraction(float(c_mean[0, j * 2 + t]))
               - Fraction(float(cb[j, i, t]))) ** 2 for t in range(2)) for i in range(16)]
         for j in range(cb.shape[0])]
    R = max(max(Tj) - min(Tj) for Tj in T)
    aa = Fraction(255) / R
    exp_Q = [[int((Tj[i] - min(Tj)) * aa + Fraction(1, 2)) for i in range(16)] for Tj in T]
    exp_b = int(sum(min(Tj) for Tj in T) * aa + Fraction(1, 2))
    assert Q[0].tolist() == exp_Q == g["Q"]
    assert int(bias[0]) == exp_b == g["bias"]
    assert abs(a - float(aa)) <= 1e-6 * float(aa)


@pytest.mark.parametrize("ip", [False, True])
def test_quantised_scan_error_bound_and_integer_sums(orc, ip):
    """|D/a - ADC| <= (M+1)/(2a) (half a quantum per table entry plus the
    bias), up to FP32 table round-off; integer sums equal a numpy gather."""
    ix, rng = tiny_index(orc, ip=ip)
    M = ix["M"]
    q = ix["X"][5] + 0.1 * rng.normal(size=ix["d"]).astype(np.float32)
    probes, _ = orc.rank(q, ix["c_rank"], ix["spherical"], 4)
    Q, bias, a = orc.lut_q8(q, ix, probes)
    assert Q.max() == 255 and np.all(Q.min(axis=2) == 0)
    for pi, p in enumerate(probes):
        mem = ix["list_ids"][ix["list_off"][p]:ix["list_off"][p + 1]]
        for i in mem[:100]:
            code = ix["codes"][i]
            D = orc.int_dist(Q[pi], bias[pi], code)
            assert D == int(bias[pi]) + int(Q[pi][np.arange(M), code].astype(np.int64).sum())
            adc = orc.adc64(q, ix, int(p), code)
            bound = (M + 1) / (2 * a) + 1e-5 * (abs(adc) + M * 255 / a)
            assert abs(D / a - adc) <= bound


# ---------------------------------------------------------------- scan + selection
def test_scan_topr_matches_library_sort(orc):
    ix, rng = tiny_index(orc)
    M = ix["M"]
    q = rng.normal(size=ix["d"]).astype(np.float32)
    probes, _ = orc.rank(q, ix["c_rank"], False, 3)
    Q, bias, _ = orc.lut_q8(q, ix, probes)
    keys = orc.scan_topr(ix, probes, Q, bias, 150)
    allk = []
    for pi, p in enumerate(probes):
        mem = ix["list_ids"][ix["list_off"][p]:ix["list_off"][p + 1]]
        D = bias[pi] + Q[pi][np.arange(M)[None, :], ix["codes"][mem]].astype(np.int64).sum(1)
        allk += [((int(Dv) + (1 << 31)) << 32) | int(i) for Dv, i in zip(D, mem)]
    ref = np.sort(np.array(allk, np.uint64))[:150]
    assert np.array_equal(keys, ref)
    assert np.array_equal(orc.key_dist(keys[:3]) >= -(1 << 31), [True] * 3)


# ---------------------------------------------------------------- rerank / knn / recall
def test_exact_knn_and_rerank_match_library(orc):
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(4)
    X = rng.integers(0, 4, size=(500, 6)).astype(np.float32)  # many exact ties
    Q = rng.integers(0, 4, size=(20, 6)).astype(np.float32)
    ids, dd = orc.exact_knn(Q, X, 10)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for qi in range(20):
        order = np.lexsort((np.arange(500), D[qi]))[:10]
        assert np.array_equal(ids[qi], order)
        np.testing.assert_array_equal(dd[qi], D[qi][order])
    ix = orc.make_index(X, X[:2], X[:2], np.zeros((2, 16, 3), np.float32),
                        np.zeros((500, 2), np.uint8), np.zeros(500, np.int32))
    cand = rng.permutation(500)[:50].astype(np.int32)
    rid, rd = orc.rerank(Q[0], ix, cand, 60)
    order = cand[np.lexsort((cand, D[0][cand]))]
    assert np.array_equal(rid[:50], order) and np.all(rid[50:] == -1) and np.all(np.isinf(rd[50:]))
    # inner product: similarity, descending, ties by id
    ixp = dict(ix, ip=True)
    rid, rd = orc.rerank(Q[0], ixp, cand, 10)
    sim = X[cand].astype(np.float64) @ Q[0].astype(np.float64)
    order = cand[np.lexsort((cand, -sim))][:10]
    assert np.array_equal(rid, order)


def test_recall_special_cases(orc):
    rng = np.random.default_rng(5)
    X = rng.normal(size=(300, 4)).astype(np.float32)
    Q = rng.normal(size=(7, 4)).astype(np.float32)
    ids, dd = orc.exact_knn(Q, X, 10)
    assert orc.recall(Q, X, ids, dd, 10) == 1.0
    far = np.argsort(-((Q[:, None] - X[None]) ** 2).sum(-1), axis=1)[:, :10]
    assert orc.recall(Q, X, far.astype(np.int64), dd, 10) == 0.0
    dup = ids.copy()
    dup[:, 1:] = dup[:, :1]  # one distinct true id per query
    assert abs(orc.recall(Q, X, dup, dd, 10) - 0.1) < 1e-12


def test_end_to_end_full_probe_full_rerank_is_exact(orc):
    """nprobe = L and R >= n: the search returns exactly the brute-force
    top-k (ties by id) and recall 1."""
    ix, rng = tiny_index(orc, n=1500)
    Q = ix["X"][rng.integers(0, 1500, 12)] + rng.normal(size=(12, ix["d"])).astype(np.float32)
    out = orc.search(ix, Q, ix["L"], 1500, 10)
    ids, dd = orc.exact_knn(Q, ix["X"], 10)
    assert np.array_equal(out["ids"], ids)
    np.testing.assert_array_equal(out["dists"], dd)
    assert orc.recall(Q, ix["X"], out["ids"], dd, 10) == 1.0


def test_small_config_recall_sane(orc):
    """The small configuration (10k x 128, L = 64, M = 64, nprobe 8, R 100)
    reaches high recall: a dropped term or a wrong sign anywhere would not."""
    X = synth.base(1)
    Q = synth.queries(1, 30)
    ix = orc.build_index(X, 64, 64, False, synth.build_perm(1, len(X)), iters=5)
    out = orc.search(ix, Q, 8, 100, 10)
    _, dd = orc.exact_knn(Q, X, 10)
    assert orc.recall(Q, X, out["ids"], dd, 10) >= 0.9


# ---------------------------------------------------------------- hybrid (Sec. 4.4)
def test_hybrid_reduces_to_full_scan_and_graph_only(orc):
    ix, rng = tiny_index(orc, n=1200, L=6)
    g, entry = orc.build_graph(ix)
    # graph: exact 32-NN inside the list (library distance + sort)
    from scipy.spatial.distance import cdist
    for c in range(2):
        mem = ix["list_ids"][ix["list_off"][c]:ix["list_off"][c + 1]]
        D = cdist(ix["X"][mem].astype(np.float64), ix["X"][mem].astype(np.float64), "sqeuclidean")
        for r, u in enumerate(mem[:20]):
            dd = D[r].copy()
            dd[r] = np.inf
            order = mem[np.lexsort((mem, dd))][:32]
            assert np.array_equal(g[u], order)
    q = rng.normal(size=ix["d"]).astype(np.float32)
    probes, _ = orc.rank(q, ix["c_rank"], False, 5)
    Q, bias, _ = orc.lut_q8(q, ix, probes)
    full = orc.scan_topr(ix, probes, Q, bias, 100)
    # tau = 0: every distant probe is scanned fully -> the plain scan
    k0, nf = orc.hybrid_topr(ix, g, entry, probes, Q, bias, 100, n_near=2, efs=64, tau=0)
    assert np.array_equal(k0, full) and nf == 5
    # efs >= every list: each distant probe's graph result is the entry's
    # reachable set (a BFS in the test); tau = infinity takes only those sets,
    # so the expectation needs no call of the oracle's graph search.
    big = int(np.diff(ix["list_off"]).max()) + 1
    kinf, nf = orc.hybrid_topr(ix, g, entry, probes, Q, bias, 10_000, n_near=2, efs=big, tau=1 << 30)
    assert nf == 2
    expect = list(full_keys(ix, probes[0], Q[0], bias[0])) + list(full_keys(ix, probes[1], Q[1], bias[1]))
    for pi in range(2, 5):
        reach = reachable(g, entry[probes[pi]])
        expect += list(member_keys(ix, reach, Q[pi], bias[pi]))
    assert np.array_equal(kinf, np.sort(np.array(expect, np.uint64)))


def reachable(g, e):
    """Nodes reachable from e along the graph's out-edges (BFS)."""
    seen, todo = {int(e)}, [int(e)]
    while todo:
        u = todo.pop()
        for v in g[u]:
            if v >= 0 and int(v) not in seen:
                seen.add(int(v))
                todo.append(int(v))
    return np.array(sorted(seen), np.int64)


def member_keys(ix, ids, Qp, bias_p):
    """Sorted candidate keys ((D + 2^31) << 32) | id of the given vectors,
    D = bias + sum_j Q[j][code_j] (Alg. 3 distance) computed with numpy."""
    ids = np.asarray(ids, np.int64)
    D = int(bias_p) + Qp[np.arange(ix["M"])[None, :], ix["codes"][ids]].astype(np.int64).sum(1)
    return np.sort(np.array([((int(a) + (1 << 31)) << 32) | int(b) for a, b in zip(D, ids)], np.uint64))


def full_keys(ix, c, Qp, bias_p):
    return member_keys(ix, ix["list_ids"][ix["list_off"][c]:ix["list_off"][c + 1]], Qp, bias_p)


def test_graph_search_large_pool_returns_the_reachable_set(orc):
    """With a result capacity efs at least the number of nodes reachable from
    the entry, best-first search (Sec. 4.4) never stops early and never
    evicts: W is exactly the reachable set. The fixture holds lists whose
    32-NN graph is connected (W = the whole list) and one whose entry reaches
    only part of it; with efs below the reachable count, |W| = efs."""
    ix, rng = tiny_index(orc, n=1200, L=6)
    g, entry = orc.build_graph(ix)
    q = rng.normal(size=ix["d"]).astype(np.float32)
    allp = np.arange(ix["L"], dtype=np.int32)
    Q, bias, _ = orc.lut_q8(q, ix, allp)
    whole = partial = 0
    for c in range(ix["L"]):
        mem = ix["list_ids"][ix["list_off"][c]:ix["list_off"][c + 1]]
        reach = reachable(g, entry[c])
        assert set(reach.tolist()) <= set(mem.tolist())
        whole += len(reach) == len(mem)
        partial += len(reach) < len(mem)
        for efs in (len(reach), len(reach) + 7):
            W = orc.graph_search(ix, g, entry[c], Q[c], bias[c], efs)
            assert np.array_equal(W, member_keys(ix, reach, Q[c], bias[c]))
        for efs in (1, 5, len(reach) // 2):
            W = orc.graph_search(ix, g, entry[c], Q[c], bias[c], efs)
            assert len(W) == min(efs, len(reach))
            assert set(orc.key_id(W).tolist()) <= set(reach.tolist())
    assert whole >= 1 and partial >= 1


# A hand-made graph with one subspace (M = 1): node i has code i, and the
# probe's table row gives node i the distance TAB[i], so every key is set by
# hand. Edges in adjacency order; -1 pads to 32 neighbours.
HAND_TAB = [50, 40, 60, 70, 30, 55, 45, 10]
HAND_EDGES = {0: [1, 2, 3], 1: [4, 5], 2: [], 3: [], 4: [6, 0], 5: [], 6: [7], 7: [6, 5]}


def hand_graph(n_extra=0):
    n = 8 + n_extra
    g = -np.ones((n, 32), np.int32)
    for u, vs in HAND_EDGES.items():
        g[u, :len(vs)] = vs
    return g


def hand_key(D, i):
    return ((D + (1 << 31)) << 32) | i


def test_graph_search_hand_trace(orc):
    """Best-first search of Sec. 4.4 traced by hand on an 8-node graph, efs 3.

    From entry 0 (50): expand 0 -> W {0:50, 1:40, 2:60}; node 3 (70) is not
    below max W, skipped. Expand 1 (40 < max 60) -> 4 (30) enters, 60 is
    evicted: W {0, 1, 4}; 5 (55) is not below 50. Expand 4 -> 6 (45) enters,
    50 evicted: W {1, 4, 6}. Pop 6: W is full and 6 is its own maximum; the
    stop test asks for a key above the maximum, so 6 is expanded -> 7 (10)
    enters, 45 evicted: W {1, 4, 7}. Expand 7 (no new node). Pop 2 (60 > 40):
    stop. Result: nodes 7, 4, 1."""
    n = 8
    ix = {"codes": np.arange(n, dtype=np.uint8)[:, None].copy(), "M": 1, "n": n}
    Qp = np.zeros((1, 16), np.uint8)
    Qp[0, :n] = HAND_TAB
    W = orc.graph_search(ix, hand_graph(), 0, Qp, 0, 3)
    assert W.tolist() == [hand_key(10, 7), hand_key(30, 4), hand_key(40, 1)]
    # efs 1: expand 0 -> 1 (40) replaces 0; pop 1 (= max W, expanded) -> 4
    # (30) replaces 1; pop 4, its new neighbour 6 (45) is not below 30; no
    # candidate is left.
    W1 = orc.graph_search(ix, hand_graph(), 0, Qp, 0, 1)
    assert W1.tolist() == [hand_key(30, 4)]
    # bias shifts every key's distance, not the order
    Wb = orc.graph_search(ix, hand_graph(), 0, Qp, -25, 3)
    assert Wb.tolist() == [hand_key(-15, 7), hand_key(5, 4), hand_key(15, 1)]


def test_hybrid_hand_example(orc):
    """The hybrid of Sec. 4.4 on hand-made lists: list 0 (nodes 8..11, near,
    distances 20, 35, 42, 90) is scanned fully; list 1 is the hand graph
    above with efs 3, whose graph result is nodes {7, 4, 1} (10, 30, 40).

    R = 2: theta = the 2nd key of the near list (35, node 9); two graph
    results lie below it, so tau = 2 scans list 1 fully and tau = 3 does not.
    R = 12: fewer than R near keys, theta = +inf, all 3 results count: tau =
    3 gives the union of both whole lists, tau = 4 the near list plus {7, 4, 1}."""
    n = 12
    codes = np.arange(n, dtype=np.uint8)[:, None].copy()
    ix = {"codes": codes, "M": 1, "n": n,
          "list_off": np.array([0, 4, 12], np.int64),
          "list_ids": np.array([8, 9, 10, 11, 0, 1, 2, 3, 4, 5, 6, 7], np.int32)}
    g = hand_graph(n_extra=4)
    entry = np.array([8, 0], np.int32)
    probes = np.array([0, 1], np.int32)
    Q = np.zeros((2, 1, 16), np.uint8)
    Q[0, 0, 8:12] = [20, 35, 42, 90]
    Q[1, 0, :8] = HAND_TAB
    bias = np.zeros(2, np.int32)
    near = [hand_key(20, 8), hand_key(35, 9), hand_key(42, 10), hand_key(90, 11)]
    graph_only = sorted(near + [hand_key(10, 7), hand_key(30, 4), hand_key(40, 1)])
    whole = sorted(near + [hand_key(d, i) for i, d in enumerate(HAND_TAB)])
    k, nf = orc.hybrid_topr(ix, g, entry, probes, Q, bias, 2, n_near=1, efs=3, tau=2)
    assert nf == 2 and k.tolist() == whole[:2]
    k, nf = orc.hybrid_topr(ix, g, entry, probes, Q, bias, 2, n_near=1, efs=3, tau=3)
    assert nf == 1 and k.tolist() == graph_only[:2]
    k, nf = orc.hybrid_topr(ix, g, entry, probes, Q, bias, 12, n_near=1, efs=3, tau=3)
    assert nf == 2 and k.tolist() == whole
    k, nf = orc.hybrid_topr(ix, g, entry, probes, Q, bias, 12, n_near=1, efs=3, tau=4)
    assert nf == 1 and k.tolist() == graph_only


# ---------------------------------------------------------------- learned part
def test_eq2_closed_form_points(orc):
    # p <= p0 -> Pmin; worked value; clamp at Pmax; non-decreasing in p
    assert orc.eq2(0.1, 8, 128, 0.2, 0.5) == 8
    # 120 * (0.6 - 0.2) * (0.6 + 0.5) = 52.8 -> ceil 53 -> 61
    assert orc.eq2(0.6, 8, 128, 0.2, 0.5) == 61
    assert orc.eq2(1.0, 8, 128, 0.0, 5.0) == 128
    vals = [orc.eq2(p, 4, 256, 0.3, 0.2) for p in np.linspace(0, 1, 101)]
    assert all(b >= a for a, b in zip(vals, vals[1:]))


def test_mlp_gradient_finite_differences(orc):
    rng = np.random.default_rng(6)
    F, H1, H2, B = 7, 5, 4, 9
    w = rng.normal(scale=0.5, size=orc.mlp_nparams(F, H1, H2))
    x = rng.normal(size=(B, F))
    y = rng.integers(0, 2, size=(B, 2)).astype(np.float64)
    loss, g = orc.mlp_grad(w, F, H1, H2, x, y)
    p = orc.mlp_forward(w, F, H1, H2, x)
    bce = -(y * np.log(p) + (1 - y) * np.log(1 - p)).sum(1).mean()
    assert abs(loss - bce) < 1e-10
    h = 1e-6
    for i in range(len(w)):
        e = np.zeros_like(w)
        e[i] = h
        num = (orc.mlp_grad(w + e, F, H1, H2, x, y)[0] - orc.mlp_grad(w - e, F, H1, H2, x, y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_adam_first_step_closed_form(orc):
    rng = np.random.default_rng(7)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    w0 = w.copy()
    orc.adam_step(w, g, m, v, 1, lr=0.01)
    # t = 1: m_hat = g, v_hat = g^2  ->  w1 = w0 - lr g / (|g| + eps)
    np.testing.assert_allclose(w, w0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_regression_mapping_endpoints_and_inverse():
    import oracle as o
    lo, hi = 4, 64
    assert o.reg_map(0.0, lo, hi) == lo and o.reg_map(1.0, lo, hi) == hi
    assert o.reg_map(-3.0, lo, hi) == lo and o.reg_map(7.0, lo, hi) == hi
    # the target of an exact setting maps back to it: 4 * 16^(1/2) = 16, 4 * 16^(1/4) = 8
    for v in (4, 8, 16, 32, 64):
        assert o.reg_map(float(o.reg_target(v, lo, hi)), lo, hi) == v
    # between grid points: the next integer up; shift and scale move u
    assert o.reg_map(0.6, lo, hi) == 22  # 4 * 16^0.6 = 21.11
    assert o.reg_map(0.5, lo, hi, a=0.25) == 32 and o.reg_map(0.5, lo, hi, b=-0.5) == 8
