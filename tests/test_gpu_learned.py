"""Learned nprobe / rerank predictor (Sec. 4.2.1-4.2.2, Eq. 2) on the GPU.

The training kernels are checked against the FP64 oracle (gradients within
1e-3 relative in max-norm), inference against the oracle's forward pass, the
adaptive search against the variable-nprobe search it drives, and the trained
predictor against fixed nprobe at equal recall.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

pytestmark = pytest.mark.gpu

F, H = 64, 64


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    return torch, ksc


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_mlp_gradients_match_fp64_oracle(env):
    torch, ksc = env
    rng = np.random.default_rng(91)
    npar = oracle.mlp_nparams(F, H, H)
    assert npar == 8450
    w = rng.normal(scale=0.2, size=npar)
    B = 300  # three CTAs, the last one ragged
    x = rng.normal(size=(B, F))
    y = rng.integers(0, 2, size=(B, 2)).astype(np.float64)
    loss_ref, g_ref = oracle.mlp_grad(w, F, H, H, x, y)
    wd = torch.tensor(w, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    g = torch.empty(npar, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert ksc.lib().ksc_mlp_grad(_ptr(wd), _ptr(xd), _ptr(yd), B, _ptr(g), _ptr(loss), st) == 0
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - loss_ref) <= 1e-5 * abs(loss_ref)
    assert np.abs(g - g_ref).max() <= 1e-3 * np.abs(g_ref).max()


def test_mlp_bf16_inference_matches_oracle_forward(env):
    torch, ksc = env
    rng = np.random.default_rng(92)
    npar = oracle.mlp_nparams(F, H, H)
    w = rng.normal(scale=0.15, size=npar)
    x = rng.normal(size=(257, F))
    ref = oracle.mlp_forward(w, F, H, H, x)
    wd = torch.tensor(w, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    p = torch.empty((257, 2), dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert ksc.lib().ksc_mlp_forward(_ptr(wd), _ptr(xd), 257, _ptr(p), st) == 0
    torch.cuda.synchronize()
    # BF16 weights / activations: about 2^-8 relative per operand
    assert np.abs(p.cpu().numpy() - ref).max() < 3e-2


def _kth(torch, X, Q, k=10, chunk=2048):
    Xd = torch.from_numpy(X).cuda().double()
    xn = (Xd * Xd).sum(1)
    out = []
    for b in range(0, len(Q), chunk):
        Qd = torch.from_numpy(Q[b:b + chunk]).cuda().double()
        D = (Qd * Qd).sum(1, keepdim=True) - 2 * Qd @ Xd.T + xn[None]
        out.append(torch.topk(D, k, dim=1, largest=False).values[:, k - 1].float())
    return torch.cat(out).contiguous()


@pytest.fixture(scope="module")
def trained(env):
    """The 1M x 128 SIFT-shaped workload, predictor trained on 30k seeded
    training queries; 2000 evaluation and 2000 validation queries."""
    torch, ksc = env
    X = synth.base(2)
    Q = synth.queries(2, 2000)
    TV = synth.train_queries(5, 32_000)
    T, Vq = TV[:30_000], TV[30_000:]
    g = ksc.build_index(torch.from_numpy(X).cuda(), 1024, 64, perm=synth.build_perm(2, len(X)))
    loss = g.train_predictor(torch.from_numpy(T).cuda(), _kth(torch, X, T), epochs=8)
    return g, X, Q, Vq, loss


def test_eq2_and_features_on_device_follow_the_oracle(env, trained):
    torch, ksc = env
    g, X, Q, Vq, loss = trained
    assert np.isfinite(loss) and loss < 1.2  # well below the 2 ln 2 of an untrained net
    g.set_predictor_params(pmin=4, pmax=64, rmin=20, rmax=400, p0=0.25, p1=0.4, r0=0.3, r1=0.6)
    Qd = torch.from_numpy(Q).cuda()
    ids, dists, npb, rr = g.search_adaptive(Qd, 10)
    feats = g.query_features(Qd)
    w = torch.tensor(g.predictor_weights(), device="cuda")
    p = torch.empty((len(Q), 2), dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert ksc.lib().ksc_mlp_forward(_ptr(w), _ptr(feats), len(Q), _ptr(p), st) == 0
    torch.cuda.synchronize()
    p = p.cpu().numpy().astype(np.float64)
    npb, rr = npb.cpu().numpy(), rr.cpu().numpy()
    ref_n = np.array([oracle.eq2(v, 4, 64, 0.25, 0.4) for v in p[:, 0]])
    ref_r = np.array([oracle.eq2(v, 20, 400, 0.3, 0.6) for v in p[:, 1]])
    # FP32 on the device, FP64 in the oracle: equal except at a ceil boundary
    assert np.abs(npb - ref_n).max() <= 1 and (npb == ref_n).mean() >= 0.99
    assert np.abs(rr - ref_r).max() <= 1 and (rr == ref_r).mean() >= 0.99
    # the search's fused head (features + network in one kernel) gives the
    # settings of the separate feature and forward kernels exactly: Eq. 2
    # evaluated in FP32 on their probabilities
    def eq2_f32(v, lo, hi, a, b):
        v = np.float32(v)
        relu = max(v - np.float32(a), np.float32(0))
        r = np.float32(lo) + np.ceil(np.float32(hi - lo) * relu * (v + np.float32(b)))
        return int(min(max(r, np.float32(lo)), np.float32(hi)))
    p32 = p.astype(np.float32)
    assert np.array_equal(npb, [eq2_f32(v, 4, 64, 0.25, 0.4) for v in p32[:, 0]])
    assert np.array_equal(rr, [eq2_f32(v, 20, 400, 0.3, 0.6) for v in p32[:, 1]])
    # features: distances of the 32 nearest lists, normalised
    f = feats.cpu().numpy()
    assert np.allclose(f[:, :32].mean(1), 1.0, atol=1e-4) and np.all(f[:, 32] > 0.999)
    assert np.all(np.diff(f[:, :32], axis=1) >= -1e-6)
    # the adaptive search is the variable-nprobe search at the predicted values
    ids2, d2 = g.search_varprobe(Qd, 10, torch.from_numpy(npb).cuda(), torch.from_numpy(rr).cuda(),
                                 nprobe_max=64, rerank_max=400)
    assert torch.equal(ids, ids2) and torch.equal(dists, d2)


def _recall(torch, X, Q, ids, kth):
    Xd = torch.from_numpy(X).cuda().double()
    Qd = torch.from_numpy(Q).cuda().double()
    idt = ids.clamp_min(0)
    d = ((Xd[idt] - Qd[:, None, :]) ** 2).sum(-1)
    hit = (d <= kth.double()[:, None] + 1e-6) & (ids >= 0)
    return float(hit.sum(1).clamp_max(10).double().mean().item() / 10)


def test_learned_nprobe_beats_fixed_nprobe_at_equal_recall(env, trained):
    """What the predictor gains: the fewest probes on average that reach
    recall@10 >= 0.90 -- fixed nprobe vs the adaptive search with Eq. 2 tuned
    on a validation split and evaluated on separate queries."""
    torch, ksc = env
    g, X, Q, Vq, _ = trained
    Qd = torch.from_numpy(Q).cuda()
    Vd = torch.from_numpy(Vq).cuda()
    kq, kv = _kth(torch, X, Q), _kth(torch, X, Vq)
    target = 0.90
    fixed = None
    for P in range(1, 65):
        ids, _ = g.search(Qd, 10, P, 200)
        if _recall(torch, X, Q, ids, kq) >= target:
            fixed = P
            break
    assert fixed is not None
    best = None
    for pmax in (16, 32, 64):
        for p0 in (0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6):
            for p1 in (0.0, 0.5, 1.0, 2.0):
                g.set_predictor_params(pmin=1, pmax=pmax, rmin=200, rmax=200, p0=p0, p1=p1, r0=0.0, r1=0.0)
                ids, _, npb, _ = g.search_adaptive(Vd, 10)
                rec = _recall(torch, X, Vq, ids, kv)
                cost = float(npb.double().mean().item())
                if rec >= target + 0.005 and (best is None or cost < best[0]):
                    best = (cost, pmax, p0, p1)
    assert best is not None, "no Eq. 2 setting reached the target recall on the validation split"
    g.set_predictor_params(pmin=1, pmax=best[1], rmin=200, rmax=200, p0=best[2], p1=best[3], r0=0.0, r1=0.0)
    ids, _, npb, _ = g.search_adaptive(Qd, 10)
    rec = _recall(torch, X, Q, ids, kq)
    mean_np = float(npb.double().mean().item())
    print("fixed nprobe %d vs learned mean nprobe %.2f at recall %.4f (pmax %d, p0 %.1f, p1 %.1f)"
          % (fixed, mean_np, rec, best[1], best[2], best[3]))
    assert rec >= target and mean_np < fixed


def test_regression_heads_follow_the_oracle_mapping_and_gain(env, trained):
    """Regression variant (soft targets, log-linear mapping): the device's
    settings equal the oracle's mapping of the same probabilities, and the
    variant also needs fewer probes than fixed nprobe at recall 0.90."""
    torch, ksc = env
    g, X, Q, Vq, _ = trained
    T = synth.train_queries(5, 32_000)[:30_000]
    loss = g.train_predictor(torch.from_numpy(T).cuda(), _kth(torch, X, T), epochs=8, regression=True)
    assert np.isfinite(loss) and loss < 2 * np.log(2)
    g.set_predictor_params(4, 64, 20, 400, 0.1, 0.2, 0.0, 0.1, regression=True)
    Qd = torch.from_numpy(Q).cuda()
    ids, dists, npb, rr = g.search_adaptive(Qd, 10)
    feats = g.query_features(Qd)
    w = torch.tensor(g.predictor_weights(), device="cuda")
    p = torch.empty((len(Q), 2), dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert ksc.lib().ksc_mlp_forward(_ptr(w), _ptr(feats), len(Q), _ptr(p), st) == 0
    torch.cuda.synchronize()
    p = p.cpu().numpy().astype(np.float64)
    npb, rr = npb.cpu().numpy(), rr.cpu().numpy()
    ref_n = np.array([oracle.reg_map(v, 4, 64, 0.1, 0.2) for v in p[:, 0]])
    ref_r = np.array([oracle.reg_map(v, 20, 400, 0.0, 0.1) for v in p[:, 1]])
    assert np.abs(npb - ref_n).max() <= 1 and (npb == ref_n).mean() >= 0.99
    assert np.abs(rr - ref_r).max() <= 1 and (rr == ref_r).mean() >= 0.99
    assert len(np.unique(npb)) > 3  # the heads spread the queries over the range
    Vd = torch.from_numpy(Vq).cuda()
    kq, kv = _kth(torch, X, Q), _kth(torch, X, Vq)
    fixed = next(P for P in range(1, 65) if _recall(torch, X, Q, g.search(Qd, 10, P, 200)[0], kq) >= 0.90)
    best = None
    for pmax in (16, 32, 64):
        for p0 in (-0.3, -0.2, -0.1, 0.0, 0.1, 0.2, 0.3):
            for p1 in (-0.5, 0.0, 0.5, 1.0):
                g.set_predictor_params(1, pmax, 200, 200, p0, p1, 0.0, 0.0, regression=True)
                vi, _, vn, _ = g.search_adaptive(Vd, 10)
                if _recall(torch, X, Vq, vi, kv) >= 0.905:
                    cost = float(vn.double().mean().item())
                    if best is None or cost < best[0]:
                        best = (cost, pmax, p0, p1)
    assert best is not None
    g.set_predictor_params(1, best[1], 200, 200, best[2], best[3], 0.0, 0.0, regression=True)
    ids, _, npb, _ = g.search_adaptive(Qd, 10)
    rec, mean_np = _recall(torch, X, Q, ids, kq), float(npb.double().mean().item())
    print("regression heads: fixed nprobe %d vs mean nprobe %.2f at recall %.4f" % (fixed, mean_np, rec))
    assert rec >= 0.90 and mean_np < fixed


def _eq2_f32(v, lo, hi, a, b):
    """Eq. 2 in FP32, operation by operation as the device evaluates it."""
    v = np.float32(v)
    relu = max(v - np.float32(a), np.float32(0))
    r = np.float32(lo) + np.ceil(np.float32(hi - lo) * relu * (v + np.float32(b)))
    return int(min(max(r, np.float32(lo)), np.float32(hi)))


@pytest.mark.parametrize("metric", ["l2", "spherical"])
def test_adaptive_ranking_equals_the_separate_head(env, metric):
    """Batches of at least 8 queries per SM rank in one kernel (32 smallest
    scores, features, network, Eq. 2, exact ranking of the predicted lists);
    smaller ones take the ranking with features, then the head kernel.  In
    both shapes, for L2 and spherical scores, the settings equal Eq. 2 in FP32
    on the probabilities of the separate feature and forward kernels, and the
    results equal the variable-nprobe search at those settings."""
    torch, ksc = env
    rng = np.random.default_rng(17 if metric == "l2" else 18)
    centres = rng.uniform(-4, 4, size=(24, 48))
    X = (centres[rng.integers(0, 24, 6000)] + rng.normal(size=(6000, 48))).astype(np.float32)
    Q = (centres[rng.integers(0, 24, 40)] + rng.normal(size=(40, 48))).astype(np.float32)
    sph = metric == "spherical"
    if sph:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    ix_o = oracle.build_index(X, 48, 24, sph, rng.permutation(6000).astype(np.int64), iters=4, ip=sph)
    g = ksc.index_import(ix_o, metric="ip" if sph else "l2", spherical=sph)
    # weights and Eq. 2 chosen so that nprobe spreads over 1..48 (all 48 lists):
    # the kernel's paths for nprobe <= 32, 33..48 and every list
    w = np.random.default_rng(99).normal(scale=0.3, size=8450).astype(np.float32)
    g.predictor_weights(set_to=w)
    g.set_predictor_params(1, 48, 50, 150, 0.05, 3.0, 0.0, 0.5)
    wd = torch.from_numpy(w).cuda()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for reps in (1, 41):  # 40 queries (CTA shapes) and 1640 (the one-kernel ranking)
        Qd = torch.from_numpy(np.tile(Q, (reps, 1))).cuda()
        ids, dists, npb, rr = g.search_adaptive(Qd, 10)
        feats = g.query_features(Qd)
        p = torch.empty((len(Qd), 2), dtype=torch.float32, device="cuda")
        assert ksc.lib().ksc_mlp_forward(_ptr(wd), _ptr(feats), len(Qd), _ptr(p), st) == 0
        torch.cuda.synchronize()
        p = p.cpu().numpy()
        npb_h, rr_h = npb.cpu().numpy(), rr.cpu().numpy()
        assert np.array_equal(npb_h, [_eq2_f32(v, 1, 48, 0.05, 3.0) for v in p[:, 0]])
        assert np.array_equal(rr_h, [_eq2_f32(v, 50, 150, 0.0, 0.5) for v in p[:, 1]])
        assert len(np.unique(npb_h)) > 10 and npb_h.min() <= 32 and npb_h.max() > 32
        ids2, d2 = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=48, rerank_max=150)
        assert torch.equal(ids, ids2) and torch.equal(dists, d2)
        assert g.last_status() == 0
