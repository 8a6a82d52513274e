"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Integer work (quantised LUTs, biases, candidate keys) must be bit-exact;
float distances within 1e-4 relative of FP64; result ids equal except where
two exact distances tie to within that tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    return torch


@pytest.fixture(scope="module")
def ksc(torch):
    from paper_2511_03298_gb300 import ksc
    return ksc


def mixture(n, d, L, seed, ip=False, nq=40):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-4, 4, size=(max(L // 2, 2), d))
    X = (centres[rng.integers(0, len(centres), n)] + rng.normal(size=(n, d))).astype(np.float32)
    Q = (centres[rng.integers(0, len(centres), nq)] + rng.normal(size=(nq, d))).astype(np.float32)
    if ip:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    return X, Q, rng.permutation(n).astype(np.int64)


_CACHE = {}


def small_index(kind):
    """Oracle-built indexes (shared with the GPU through import)."""
    if kind not in _CACHE:
        if kind == "l2":
            X, Q, perm = mixture(6000, 64, 24, 11)
            ix = oracle.build_index(X, 24, 32, False, perm, iters=6)
        elif kind == "ip":
            X, Q, perm = mixture(5000, 48, 20, 12, ip=True)
            ix = oracle.build_index(X, 20, 24, True, perm, iters=6, ip=True)
        elif kind == "m50":  # d = 100, M = 50: subspaces not a multiple of the lane group
            X, Q, perm = mixture(4000, 100, 16, 13, ip=True)
            ix = oracle.build_index(X, 16, 50, True, perm, iters=5, ip=True)
        elif kind == "ds4":  # d' = 4: the table kernels' general sub-vector path
            X, Q, perm = mixture(3000, 64, 12, 14)
            ix = oracle.build_index(X, 12, 16, False, perm, iters=5)
        elif kind == "ds3ip":  # d' = 3, inner product
            X, Q, perm = mixture(3000, 36, 10, 15, ip=True)
            ix = oracle.build_index(X, 10, 12, True, perm, iters=5, ip=True)
        elif kind == "m48":  # d = 96, M = 48: six subspaces per lane at 8 lanes per query
            X, Q, perm = mixture(5000, 96, 20, 16, ip=True)
            ix = oracle.build_index(X, 20, 48, True, perm, iters=5)
        elif kind == "small":  # the 10k x 128 configuration
            X = synth.base(1)
            Q = synth.queries(1)
            ix = oracle.build_index(X, 64, 64, False, synth.build_perm(1, len(X)), iters=20)
        _CACHE[kind] = (ix, Q)
    return _CACHE[kind]


def gpu_index(ksc, ix):
    return ksc.index_import(ix, metric="ip" if ix["ip"] else "l2", spherical=ix["spherical"])


def oracle_probes(ix, Q, P):
    return np.stack([oracle.rank(q, ix["c_rank"], ix["spherical"], P)[0] for q in Q]).astype(np.int32)


def check_results(ix, Q, ids, dists, ref_ids, ref_d, k):
    """Tie-aware comparison of top-k results against the oracle."""
    ip = ix["ip"]
    X = ix["X"].astype(np.float64)
    for qi in range(len(Q)):
        np.testing.assert_allclose(dists[qi], ref_d[qi], rtol=RTOL, atol=1e-4)
        for r in range(k):
            if ids[qi, r] == ref_ids[qi, r]:
                continue
            assert ids[qi, r] >= 0 and ref_ids[qi, r] >= 0, (qi, r)
            x = X[ids[qi, r]]
            q = Q[qi].astype(np.float64)
            exact = -(q @ x) if ip else ((q - x) ** 2).sum()
            expect = -ref_d[qi, r] if ip else ref_d[qi, r]
            assert abs(exact - expect) <= RTOL * max(1.0, abs(expect)), (qi, r, exact, expect)


@pytest.mark.parametrize("kind", ["l2", "ip", "m50", "ds4", "ds3ip"])
def test_luts_bit_exact(torch, ksc, kind):
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    P = 7
    probes = oracle_probes(ix, Q, P)
    lut, bias, scale = g.compute_luts(torch.from_numpy(Q).cuda(), torch.from_numpy(probes).cuda())
    lut, bias, scale = lut.cpu().numpy(), bias.cpu().numpy(), scale.cpu().numpy()
    for qi in range(len(Q)):
        Ql, b, a = oracle.lut_q8(Q[qi], ix, probes[qi])
        assert np.array_equal(lut[qi], Ql), qi
        assert np.array_equal(bias[qi], b), qi
        assert np.float32(a) == scale[qi], qi


def test_luts_of_a_misaligned_query_matrix(torch, ksc):
    """A query matrix at a 4-byte (not 8-byte) offset takes the tables' general
    path; the tables are the same."""
    ix, Q = small_index("l2")
    g = gpu_index(ksc, ix)
    probes = torch.from_numpy(oracle_probes(ix, Q, 7)).cuda()
    Qa = torch.from_numpy(Q).cuda()
    buf = torch.empty(Q.size + 1, dtype=torch.float32, device="cuda")
    Qm = buf[1:].view(Q.shape)
    Qm.copy_(Qa)
    assert Qm.data_ptr() % 8 == 4
    a = g.compute_luts(Qa, probes)
    b = g.compute_luts(Qm, probes)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    s1 = g.search_with_probes(Qa, probes, 10, 100)
    s2 = g.search_with_probes(Qm, probes, 10, 100)
    for x, y in zip(s1, s2):
        assert torch.equal(x, y)


@pytest.mark.parametrize("kind,lanes", [("l2", 4), ("l2", 8), ("l2", 16), ("l2", 32), ("ip", 4), ("ip", 8),
                                        ("ip", 32), ("m50", 4), ("m50", 8), ("m50", 16), ("m50", 32), ("small", 0),
                                        ("small", 4), ("ds4", 4), ("ds4", 8), ("ds3ip", 4), ("ds3ip", 16)])
def test_scan_candidates_bit_exact(torch, ksc, kind, lanes):
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    P, R, k = (8, 100, 10) if kind == "small" else (5, 150, 10)
    probes = oracle_probes(ix, Q, P)
    opts = ksc.search_opts(lanes_per_query=lanes)
    ids, dists, cand, ncand = g.search_with_probes(torch.from_numpy(Q).cuda(), torch.from_numpy(probes).cuda(),
                                                   k, R, opts=opts)
    cand = cand.cpu().numpy().view(np.uint64)
    ncand = ncand.cpu().numpy()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    ref_ids = np.zeros_like(ids)
    ref_d = np.zeros(ids.shape, np.float64)
    for qi in range(len(Q)):
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, probes[qi])
        ref = oracle.scan_topr(ix, probes[qi], Ql, b, R)
        assert ncand[qi] == len(ref)
        assert np.array_equal(cand[qi, :len(ref)], ref), qi
        ref_ids[qi], ref_d[qi] = oracle.rerank(Q[qi], ix, oracle.key_id(ref).astype(np.int32), k)
    check_results(ix, Q, ids, dists, ref_ids, ref_d, k)
    assert g.last_status() == 0


@pytest.mark.parametrize("kind,lanes", [("l2", 0), ("l2", 16), ("m48", 0), ("m50", 8), ("ip", 8)])
@pytest.mark.parametrize("nq", [1, 2, 3, 5])
def test_scan_sparse_lists_bit_exact(torch, ksc, kind, lanes, nq):
    """Few queries, so most lists are probed by fewer queries than a warp has
    query slots: the slots of such an item split its blocks.  Candidates equal
    the oracle's bit for bit (both scan parts: the nearest lists without a
    filter, the rest against the threshold)."""
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    Qs = Q[:nq]
    P, R, k = 9, 150, 10
    probes = oracle_probes(ix, Qs, P)
    opts = ksc.search_opts(lanes_per_query=lanes)
    for tb in (0, 3):
        opts.tile_blocks = tb
        _, _, cand, ncand = g.search_with_probes(torch.from_numpy(Qs).cuda(), torch.from_numpy(probes).cuda(),
                                                 k, R, opts=opts)
        cand = cand.cpu().numpy().view(np.uint64)
        ncand = ncand.cpu().numpy()
        for qi in range(nq):
            Ql, b, _ = oracle.lut_q8(Qs[qi], ix, probes[qi])
            ref = oracle.scan_topr(ix, probes[qi], Ql, b, R)
            assert ncand[qi] == len(ref)
            assert np.array_equal(cand[qi, :len(ref)], ref), (qi, tb)
    assert g.last_status() == 0


@pytest.mark.parametrize("kind", ["l2", "ip", "small"])
def test_rank_lists_within_fp32_tolerance(torch, ksc, kind):
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    P = 9
    probes, scores = g.rank_lists(torch.from_numpy(Q).cuda(), P)
    probes, scores = probes.cpu().numpy(), scores.cpu().numpy()
    C = ix["c_rank"].astype(np.float64)
    for qi, q in enumerate(Q.astype(np.float64)):
        ref, ref_s = oracle.rank(Q[qi], ix["c_rank"], ix["spherical"], P)
        exact = -(C @ q) if ix["spherical"] else ((C - q) ** 2).sum(1)
        tol = 1e-5 * (np.abs(q) @ np.abs(C).max(0) + (q ** 2).sum() + (C ** 2).sum(1).max())
        assert len(set(probes[qi])) == P
        # every returned list is within rounding of the oracle's P-th score
        assert np.all(exact[probes[qi]] <= ref_s[-1] + tol)
        np.testing.assert_allclose(scores[qi], exact[probes[qi]], rtol=1e-4, atol=tol)
        # the same list at every rank, except where two lists' exact scores
        # are within rounding of each other (an FP32 near-tie may swap them)
        same = probes[qi] == ref
        assert np.all(same | (np.abs(exact[probes[qi]] - exact[ref]) <= 2 * tol)), (qi, probes[qi], ref)


@pytest.mark.parametrize("kind", ["l2", "ip", "small"])
def test_search_end_to_end_matches_oracle(torch, ksc, kind):
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    P, R, k = (8, 100, 10) if kind == "small" else (6, 120, 10)
    ids, dists = g.search(torch.from_numpy(Q).cuda(), k, P, R)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    out = oracle.search(ix, Q, P, R, k)
    _, true_d = oracle.exact_knn(Q, ix["X"], k, ip=ix["ip"])
    r_gpu = oracle.recall(Q, ix["X"], ids, true_d, k, ip=ix["ip"])
    r_orc = oracle.recall(Q, ix["X"], out["ids"], true_d, k, ip=ix["ip"])
    assert abs(r_gpu - r_orc) <= 0.002
    if kind == "small":
        assert r_gpu >= 0.9
    check_results(ix, Q, ids, dists, out["ids"], out["dists"], k)


def test_full_probe_full_rerank_equals_brute_force(torch, ksc):
    ix, Q = small_index("l2")
    g = gpu_index(ksc, ix)
    k = 10
    ids, dists = g.search(torch.from_numpy(Q[:8]).cuda(), k, ix["L"], 4096)
    ref_ids, ref_d = oracle.exact_knn(Q[:8], ix["X"], k)
    check_results(ix, Q[:8], ids.cpu().numpy(), dists.cpu().numpy(), ref_ids, ref_d, k)


def test_candidate_store_overflow_is_redone_exactly(torch, ksc):
    ix, Q = small_index("l2")
    g = gpu_index(ksc, ix)
    P, R, k = 6, 100, 10
    probes = oracle_probes(ix, Q, P)
    opts = ksc.search_opts(cand_cap=R)  # far too small: every query overflows
    _, _, cand, _ = g.search_with_probes(torch.from_numpy(Q).cuda(), torch.from_numpy(probes).cuda(), k, R,
                                         opts=opts)
    assert g.last_status() & ksc.STATUS_CAND_OVERFLOW
    cand = cand.cpu().numpy().view(np.uint64)
    for qi in range(0, len(Q), 5):
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, probes[qi])
        assert np.array_equal(cand[qi], oracle.scan_topr(ix, probes[qi], Ql, b, R))


def test_short_results_padding_and_empty_batch(torch, ksc):
    X, Q, perm = mixture(300, 16, 4, 21, nq=5)
    ix = oracle.build_index(X, 4, 8, False, perm, iters=3)
    g = gpu_index(ksc, ix)
    # one probe of ~75 vectors, R = 500, k = 200: fewer than k candidates
    ids, dists = g.search(torch.from_numpy(Q).cuda(), 200, 1, 500)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    out = oracle.search(ix, Q, 1, 500, 200)
    assert np.array_equal(ids == -1, out["ids"] == -1)
    assert np.all(np.isinf(dists[ids == -1]))
    e_ids, e_d = g.search(torch.zeros((0, 16), device="cuda"), 10, 2, 50)
    assert e_ids.shape == (0, 10)


def test_varprobe_matches_oracle(torch, ksc):
    ix, Q = small_index("l2")
    g = gpu_index(ksc, ix)
    rng = np.random.default_rng(31)
    npb = rng.integers(1, 12, size=len(Q)).astype(np.int32)
    rr = rng.integers(10, 200, size=len(Q)).astype(np.int32)
    k = 10
    ids, dists = g.search_varprobe(torch.from_numpy(Q).cuda(), k, torch.from_numpy(npb).cuda(),
                                   torch.from_numpy(rr).cuda())
    out = oracle.search(ix, Q, npb, rr, k)
    check_results(ix, Q, ids.cpu().numpy(), dists.cpu().numpy(), out["ids"], out["dists"], k)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_gpu_build_index_against_oracle(torch, ksc, metric):
    """GPU build (FP32): assignments are the lowest ranking score and codes
    the nearest codewords, except where two candidates tie within FP32
    rounding; mean centroids are the member means."""
    ip = metric == "ip"
    X, Q, perm = mixture(8000, 32, 16, 41, ip=ip)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 16, 16, metric=metric, spherical=ip, perm=perm, iters=8)
    e = g.export()
    C = e["c_rank"].astype(np.float64)
    Xd = X.astype(np.float64)
    s = -(Xd @ C.T) if ip else ((Xd[:, None, :] - C[None]) ** 2).sum(-1)
    best = s[np.arange(len(X)), e["assign"]]
    assert np.all(best <= s.min(1) + 1e-5 * (1 + np.abs(s).max(1)))
    for c in range(16):
        mem = X[e["assign"] == c]
        if len(mem):
            np.testing.assert_allclose(e["c_mean"][c], mem.astype(np.float64).mean(0), rtol=1e-4, atol=1e-5)
    Rres = X - e["c_mean"][e["assign"]]
    codes, gap = oracle.encode(Rres, 16, e["codebook"])
    bad = codes != e["codes"]
    assert np.all(gap[bad] <= 1e-5 * (1 + (Rres.reshape(len(X), 16, -1) ** 2).sum(-1)[bad]))
    assert bad.mean() < 1e-3
    # the exported index searches like the oracle on the same index
    ix = oracle.make_index(X, e["c_rank"], e["c_mean"], e["codebook"], e["codes"], e["assign"], ip=ip,
                           spherical=ip)
    ids, dists = g.search(torch.from_numpy(Q).cuda(), 10, 4, 100)
    out = oracle.search(ix, Q, 4, 100, 10)
    _, true_d = oracle.exact_knn(Q, X, 10, ip=ip)
    assert abs(oracle.recall(Q, X, ids.cpu().numpy(), true_d, 10, ip=ip)
               - oracle.recall(Q, X, out["ids"], true_d, 10, ip=ip)) <= 0.002


def test_full_size_sift_sampled_parity(torch, ksc):
    """1M x 128 workload in the benchmark's launch configuration (10k queries,
    nprobe 32, R 200): candidates of sampled queries bit-exact against the
    oracle on the same (GPU-built, exported) index and probes."""
    X = synth.base(2)
    Q = synth.queries(2)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 1024, 64, perm=synth.build_perm(2, len(X)))
    e = g.export()
    ix = oracle.make_index(X, e["c_rank"], e["c_mean"], e["codebook"], e["codes"], e["assign"])
    P, R, k = 32, 200, 10
    Qd = torch.from_numpy(Q).cuda()
    gp, _ = g.rank_lists(Qd, P, want_scores=False)
    gp = gp.cpu().numpy()
    ids, dists, cand, ncand = g.search_with_probes(Qd, torch.from_numpy(gp).cuda(), k, R)
    cand = cand.cpu().numpy().view(np.uint64)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    sample = np.random.default_rng(7).choice(len(Q), 40, replace=False)
    ref_ids = np.zeros((len(sample), k), np.int64)
    ref_d = np.zeros((len(sample), k))
    for i, qi in enumerate(sample):
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, gp[qi])
        ref = oracle.scan_topr(ix, gp[qi], Ql, b, R)
        assert np.array_equal(cand[qi], ref), qi
        ref_ids[i], ref_d[i] = oracle.rerank(Q[qi], ix, oracle.key_id(ref).astype(np.int32), k)
    check_results(ix, Q[sample], ids[sample], dists[sample], ref_ids, ref_d, k)
    # the GPU ranking agrees with the FP64 ranking up to FP32 near-ties
    for qi in sample[:10]:
        ref, ref_s = oracle.rank(Q[qi], ix["c_rank"], False, P)
        assert len(np.intersect1d(ref, gp[qi])) >= P - 2


@pytest.mark.parametrize("kind", ["small", "ip", "m50"])
def test_tensor_core_list_scores_within_their_bound(torch, ksc, kind):
    """tcgen05 BF16 scores stay within the per-query bound the ranking uses."""
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    s_tc, err = g.list_scores(torch.from_numpy(Q).cuda(), tensor_cores=True)
    s_tc, err = s_tc.cpu().numpy().astype(np.float64), err.cpu().numpy().astype(np.float64)
    C = ix["c_rank"].astype(np.float64)
    Qd = Q.astype(np.float64)
    exact = -(Qd @ C.T) if ix["spherical"] else (C * C).sum(1)[None] - 2.0 * (Qd @ C.T)
    assert np.all(np.abs(s_tc - exact) <= err[:, None])
    # and they are BF16-accurate, not garbage: mean error far below the bound
    assert np.abs(s_tc - exact).mean() < 0.25 * err.mean()
    s32, err32 = g.list_scores(torch.from_numpy(Q).cuda(), tensor_cores=False)
    assert np.all(np.abs(s32.cpu().numpy() - exact) <= err32.cpu().numpy()[:, None])


@pytest.mark.parametrize("kind", ["small", "ip", "m50"])
def test_tensor_core_ranking_equals_fp32_ranking(torch, ksc, kind):
    """Both score paths re-score every list their bound cannot exclude in
    exact FP32, so the chosen probes -- and hence the results -- coincide."""
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    Qd = torch.from_numpy(Q).cuda()
    a = g.search(Qd, 10, 9, 100)
    b = g.search(Qd, 10, 9, 100, opts=ksc.search_opts(rank_fp32=True))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def e4m3_rows(torch, A):
    """Rows of A scaled by 2^(e - 8) (e: the exponent of the row's largest
    magnitude, frexp convention) and rounded to FP8 e4m3 by torch; returns
    the rounded rows (in FP64, times their scale) -- the arithmetic the FP8
    ranking option is specified to do, written with library routines."""
    A = A.astype(np.float64)
    mx = np.abs(A).max(1)
    e = np.frexp(mx)[1]
    s = np.where(mx > 0, np.ldexp(1.0, e - 8), 1.0)
    q = torch.from_numpy(A / s[:, None]).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    return q * s[:, None]


@pytest.mark.parametrize("kind", ["l2", "ip", "small", "m50"])
def test_fp8_list_scores_within_their_bound(torch, ksc, kind):
    """tcgen05 kind::f8f6f4 scores (e4m3 operands, per-row power-of-two
    scales) equal the FP64 product of the same e4m3-rounded rows up to FP32
    accumulation, and stay within the per-query bound the ranking uses."""
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    s8, err = g.list_scores(torch.from_numpy(Q).cuda(), tensor_cores=2)
    s8, err = s8.cpu().numpy().astype(np.float64), err.cpu().numpy().astype(np.float64)
    C = ix["c_rank"].astype(np.float64)
    Qd = Q.astype(np.float64)
    cn = (C * C).sum(1)
    exact = -(Qd @ C.T) if ix["spherical"] else cn[None] - 2.0 * (Qd @ C.T)
    assert np.all(np.abs(s8 - exact) <= err[:, None])
    dot8 = e4m3_rows(torch, Q) @ e4m3_rows(torch, ix["c_rank"]).T
    emu = -dot8 if ix["spherical"] else cn[None].astype(np.float32).astype(np.float64) - 2.0 * dot8
    scale = np.abs(Qd).sum(1)[:, None] * np.abs(C).max() * 4.0 + 1e-6
    assert np.all(np.abs(s8 - emu) <= 1e-5 * scale + 1e-6 * np.abs(emu))


@pytest.mark.parametrize("kind", ["l2", "small", "ip", "m50"])
def test_fp8_ranking_equals_fp32_ranking(torch, ksc, kind):
    """The FP8 scores' band is re-scored in exact FP32 like the 16-bit one:
    the probes and the results equal those of the FP32 ranking, also through
    the per-query-nprobe path."""
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    Qd = torch.from_numpy(Q).cuda()
    a = g.search(Qd, 10, 9, 100, opts=ksc.search_opts(rank_fp8=True))
    b = g.search(Qd, 10, 9, 100, opts=ksc.search_opts(rank_fp32=True))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    npb = torch.from_numpy(np.random.default_rng(3).integers(1, 12, len(Q)).astype(np.int32)).cuda()
    rr = torch.full((len(Q),), 100, dtype=torch.int32, device="cuda")
    c = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=12, rerank_max=100, opts=ksc.search_opts(rank_fp8=True))
    d = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=12, rerank_max=100, opts=ksc.search_opts(rank_fp32=True))
    assert torch.equal(c[0], d[0]) and torch.equal(c[1], d[1])
    assert g.last_status() == 0


def test_warp_shaped_kernels_bit_exact(torch, ksc):
    """Batches of at least 8 queries per SM take the warp-per-query threshold,
    select, ranking and re-rank kernels; smaller ones the CTA-per-query ones.
    Both give the oracle's candidates, and a query's result does not depend on
    which shape served it."""
    ix, Q = small_index("l2")
    g = gpu_index(ksc, ix)
    reps = 1600 // len(Q) + 1
    Qb = np.tile(Q, (reps, 1))
    P, R, k = 5, 150, 10
    probes = oracle_probes(ix, Q, P)
    pb = np.tile(probes, (reps, 1))
    big = g.search_with_probes(torch.from_numpy(Qb).cuda(), torch.from_numpy(pb).cuda(), k, R)
    small = g.search_with_probes(torch.from_numpy(Q).cuda(), torch.from_numpy(probes).cuda(), k, R)
    cand_b = big[2].cpu().numpy().view(np.uint64)
    for qi in range(len(Q)):
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, probes[qi])
        ref = oracle.scan_topr(ix, probes[qi], Ql, b, R)
        assert np.array_equal(cand_b[qi, :len(ref)], ref), qi
        assert np.array_equal(cand_b[qi + len(Q) * (reps - 1)], cand_b[qi])
    for x, y in zip(small, big):
        assert torch.equal(x, y[:len(Q)])
    # ranking: the warp and CTA shapes return the same lists
    pr_b, sc_b = g.rank_lists(torch.from_numpy(Qb).cuda(), 9)
    pr_s, sc_s = g.rank_lists(torch.from_numpy(Q).cuda(), 9)
    assert torch.equal(pr_b[:len(Q)], pr_s)


def test_tied_list_scores_take_the_general_selection(torch, ksc):
    """All but ten lists get the same ranking centroid, so their scores tie
    exactly: more than 64 scores then fall at or below the warp kernels' small
    selection bound and they fall back to radix refinement (and queries with
    more than 128 lists inside the re-score bound to the CTA kernel).  The
    warp-shaped ranking (a batch of 1600) equals the CTA-shaped one (the same
    40 queries alone) and the oracle's lists (ties by list id), and the
    adaptive search, whose one-kernel ranking takes the same fallbacks,
    equals the variable-nprobe search at its own settings."""
    X, Q, perm = mixture(8000, 32, 128, 31)
    ix = dict(oracle.build_index(X, 128, 16, False, perm, iters=3))
    cr = ix["c_rank"].copy()
    cr[10:] = cr[10]
    ix["c_rank"] = cr
    g = gpu_index(ksc, ix)
    reps = 1600 // len(Q) + 1
    Qd = torch.from_numpy(np.tile(Q, (reps, 1))).cuda()
    for P in (7, 32, 40):
        pr_b, _ = g.rank_lists(Qd, P)
        pr_s, _ = g.rank_lists(torch.from_numpy(Q).cuda(), P)
        assert torch.equal(pr_b[:len(Q)], pr_s)
        assert torch.equal(pr_b[-len(Q):], pr_s)
        ref = oracle_probes(ix, Q, P)
        # the tied lists' exact scores are identical in FP32 and FP64; the ten
        # others may reorder against them only within FP32 rounding
        same = (pr_s.cpu().numpy() == ref).mean()
        assert same >= 0.95, same
    rng = np.random.default_rng(5)
    g.predictor_weights(set_to=rng.normal(scale=0.3, size=8450))
    g.set_predictor_params(1, 40, 50, 100, 0.0, 0.0, 0.0, 0.0)
    ids, dists, npb, rr = g.search_adaptive(Qd, 10)
    assert len(np.unique(npb.cpu().numpy())) > 3
    ids2, d2 = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=40, rerank_max=100)
    assert torch.equal(ids, ids2) and torch.equal(dists, d2)
    assert g.last_status() == 0


def byte_index():
    """The 10k x 128 set mapped onto integer coordinates in [0, 255]: rows
    12 x + 128 rounded and clipped, centroids and codebooks mapped with them
    (so the codes still encode the rows), queries 12 q + 128."""
    ix, Q = small_index("small")
    X = np.clip(np.rint(12.0 * np.asarray(ix["X"], np.float64) + 128.0), 0, 255).astype(np.float32)
    assert X.min() >= 0 and X.max() <= 255 and np.all(X == np.rint(X))
    out = dict(ix, X=X, c_rank=(12.0 * np.asarray(ix["c_rank"], np.float64) + 128.0).astype(np.float32),
               c_mean=(12.0 * np.asarray(ix["c_mean"], np.float64) + 128.0).astype(np.float32),
               codebook=(12.0 * np.asarray(ix["codebook"], np.float64)).astype(np.float32))
    return out, (12.0 * np.asarray(Q, np.float64) + 128.0).astype(np.float32)


@pytest.mark.parametrize("kind", ["l2", "ip", "m50", "small", "bytes"])
def test_band_rerank_equals_fp32_rerank(torch, ksc, kind):
    """The exact re-rank's band (U8 or BF16 rows bound every candidate's FP32
    distance; only candidates whose lower bound reaches the k-th upper bound
    are read in FP32) returns what reading every candidate in FP32 returns,
    for L2 and inner products, several k and R, a fixed and a per-query R,
    in the warp-per-query shape (1600 queries); rows of real values (d = 64,
    48, 100, 128: BF16 rows) and rows of integers in [0, 255] (U8 rows, exact,
    whose band is the FP32 evaluation term alone)."""
    ix, Q = byte_index() if kind == "bytes" else small_index(kind)
    g = gpu_index(ksc, ix)
    reps = 1600 // len(Q) + 1
    Qd = torch.from_numpy(np.tile(Q, (reps, 1))).cuda()
    on, off = ksc.search_opts(rerank_band=1), ksc.search_opts(rerank_band=-1)
    for k, R in ((10, 100), (32, 200), (1, 40)):
        a = g.search(Qd, k, 9, R, opts=on)
        b = g.search(Qd, k, 9, R, opts=off)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), (k, R)
    rng = np.random.default_rng(4)
    npb = torch.from_numpy(rng.integers(1, 12, len(Qd)).astype(np.int32)).cuda()
    rr = torch.from_numpy(rng.integers(10, 150, len(Qd)).astype(np.int32)).cuda()
    c = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=12, rerank_max=150, opts=on)
    d = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=12, rerank_max=150, opts=off)
    assert torch.equal(c[0], d[0]) and torch.equal(c[1], d[1])
    assert g.last_status() == 0


@pytest.mark.parametrize("bump", ["frac", "256", "neg"])
def test_band_on_rows_that_do_not_fit_bytes(torch, ksc, bump):
    """Integer rows with a few coordinates moved out of what a byte holds (a
    fraction 0.3 that BF16 cannot hold either, the value 256, the value -1)
    take the BF16 band, with a rounding-error bound of 0 for the rows BF16
    still holds exactly; the results are still those of the FP32 re-rank."""
    ix, Q = byte_index()
    rng = np.random.default_rng({"frac": 21, "256": 22, "neg": 23}[bump])
    X = np.array(ix["X"], dtype=np.float32, copy=True)
    rows = rng.choice(len(X), 300, replace=False)
    cols = rng.integers(0, X.shape[1], len(rows))
    X[rows, cols] = {"frac": X[rows, cols] + 0.3, "256": 256.0, "neg": -1.0}[bump]
    g = gpu_index(ksc, dict(ix, X=X))
    Qd = torch.from_numpy(np.tile(Q, (1600 // len(Q) + 1, 1))).cuda()
    on, off = ksc.search_opts(rerank_band=1), ksc.search_opts(rerank_band=-1)
    for k, R in ((10, 100), (32, 200)):
        a = g.search(Qd, k, 9, R, opts=on)
        b = g.search(Qd, k, 9, R, opts=off)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), (bump, k, R)
    assert g.last_status() == 0
