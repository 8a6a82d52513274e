"""Precision variant: BF16 / FP8-e4m3 (per-row scale) first re-rank of a
widened shortlist, then the exact FP32 re-rank of its best R_f.

- R_f = R_w: identical results to the FP32 re-rank of R_w (only the order of
  the first pass differs).
- per result, the low-precision distances stay within the rounding bound of
  their row format (the errors against FP64 are printed per precision).
- recall of the widened low-precision path is within 0.01 of the FP32 path.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    return torch, ksc


def _data(ip, n=20000, d=100, nq=64, seed=5):
    rng = np.random.default_rng(seed)
    centres = rng.normal(size=(40, d))
    X = (centres[rng.integers(0, 40, n)] + 0.6 * rng.normal(size=(n, d))).astype(np.float32)
    Q = (centres[rng.integers(0, 40, nq)] + 0.6 * rng.normal(size=(nq, d))).astype(np.float32)
    if ip:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    return X, Q, rng.permutation(n).astype(np.int64)


@pytest.fixture(scope="module", params=["l2", "ip"])
def idx(env, request):
    torch, ksc = env
    ip = request.param == "ip"
    X, Q, perm = _data(ip)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 64, 50, metric=request.param, spherical=ip, perm=perm, iters=8)
    return g, X, Q, ip


@pytest.mark.parametrize("prec", [1, 2])
def test_full_final_rerank_equals_fp32(env, idx, prec):
    torch, ksc = env
    g, X, Q, ip = idx
    Qd = torch.from_numpy(Q).cuda()
    ref = g.search(Qd, 10, 8, 300)
    got = g.search(Qd, 10, 8, 300, opts=ksc.search_opts(precision=prec, rerank_final=300))
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])


def test_per_result_error_within_the_row_format_bound(env, idx):
    torch, ksc = env
    g, X, Q, ip = idx
    Qd = torch.from_numpy(Q).cuda()
    ids, _ = g.search(Qd, 100, 8, 400)
    Xd = X.astype(np.float64)
    ids_h = ids.cpu().numpy()
    qd = Q.astype(np.float64)
    rows = Xd[ids_h]                                      # [nq, c, d]
    exact = (np.einsum("qd,qcd->qc", qd, rows) if ip else ((rows - qd[:, None, :]) ** 2).sum(-1))
    qn = np.linalg.norm(qd, axis=1)[:, None]
    xn = np.linalg.norm(rows, axis=2)
    dn = np.linalg.norm(rows - qd[:, None, :], axis=2)
    xmax = np.abs(rows).max(2)
    d = X.shape[1]
    for prec, name in ((0, "fp32"), (1, "bf16"), (2, "fp8-e4m3")):
        got = g.pair_distances(Qd, ids, prec).cpu().numpy().astype(np.float64)
        err = np.abs(got - exact)
        if prec == 0:
            u, absx = 0.0, 0.0
        elif prec == 1:
            u, absx = 2.0 ** -8, 0.0
        else:  # e4m3: 3 fraction bits, subnormal spacing 2^-9 of the row scale max|x| / 448
            u, absx = 2.0 ** -4, 2.0 ** -10 * xmax / 448.0
        dx = u * xn + absx * np.sqrt(d)                   # bound on ||x_hat - x||
        acc = (d + 4) * 2.0 ** -23
        if ip:
            bound = qn * dx + acc * qn * xn
        else:
            bound = 2 * dn * dx + dx ** 2 + acc * (dn + dx) ** 2
        assert np.all(err <= bound * 1.01 + 1e-6), name
        scale = qn * xn
        print("%s: max |err| / (|q||x|) = %.3g, mean = %.3g" % (name, (err / scale).max(), (err / scale).mean()))


def test_widened_low_precision_recall(env, idx):
    torch, ksc = env
    g, X, Q, ip = idx
    Qd = torch.from_numpy(Q).cuda()
    _, true_d = oracle.exact_knn(Q, X, 10, ip=ip)
    base = g.search(Qd, 10, 8, 200)[0].cpu().numpy()
    r0 = oracle.recall(Q, X, base, true_d, 10, ip=ip)
    for prec in (1, 2):
        ids = g.search(Qd, 10, 8, 400, opts=ksc.search_opts(precision=prec, rerank_final=50))[0].cpu().numpy()
        r = oracle.recall(Q, X, ids, true_d, 10, ip=ip)
        assert r >= r0 - 0.01, (prec, r, r0)
