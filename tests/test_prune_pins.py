"""Pins of the cluster-pruning oracle (Sec. 4.2.3, Table 4, Alg. 2 f_prune).

Each function is checked against something other than itself: library
routines (numpy norms / moments / searchsorted, numpy eigh, torch layers),
closed-form values of a hand-made 2-D example, and invariants.
"""
import math

import numpy as np
import pytest

import oracle


def _lists(rng, d, sizes, spread):
    X, assign, c = [], [], []
    for p, n in enumerate(sizes):
        mu = rng.normal(size=d) * 20
        pts = mu + rng.normal(size=(n, d)) * spread
        X.append(pts)
        assign += [p] * n
        c.append(pts.mean(0) if n else mu)
    X = np.concatenate([x for x in X if len(x)]).astype(np.float32)
    return X, np.array(assign, np.int32), np.array(c, np.float32)


def test_stats_match_library_moments_and_histogram():
    rng = np.random.default_rng(1)
    d = 6
    sizes = [40, 0, 1, 25, 60]
    X, assign, c = _lists(rng, d, sizes, np.array([2.0, 1.5, 1.0, 1.0, 0.5, 0.5]))
    st, vec = oracle.prune_stats(X, c, assign)
    for p, n in enumerate(sizes):
        if n == 0:
            assert not st[p].any() and not vec[p].any()
            continue
        r = X[assign == p].astype(np.float64) - c[p].astype(np.float64)
        dist = np.linalg.norm(r, axis=1)
        rho, mu, sd = dist.max(), dist.mean(), dist.std()
        np.testing.assert_allclose(st[p, :4], [n, rho, mu, sd], rtol=1e-12, atol=1e-12)
        # bins [0, rho/4], (rho/4, rho/2], (rho/2, 3 rho/4], (3 rho/4, rho]
        b = np.searchsorted([0.25 * rho, 0.5 * rho, 0.75 * rho], dist, side="left")
        np.testing.assert_allclose(st[p, 4:8], np.bincount(b, minlength=4) / n, atol=1e-15)
        out = dist > mu + 2 * sd
        assert st[p, 8] == pytest.approx(out.mean())
        od = r[out].mean(0) if out.any() else np.zeros(d)
        np.testing.assert_allclose(vec[p, 2], od, rtol=1e-12, atol=1e-12)
        assert st[p, 11] == 0.0


def test_outlier_fraction_and_direction_on_a_planted_outlier():
    # nine members at distance 1 around the origin and one at distance 10:
    # mean 1.9, std 2.7, threshold 7.3 -> exactly one outlier
    d = 2
    ang = np.linspace(0, 2 * np.pi, 9, endpoint=False)
    pts = np.stack([np.cos(ang), np.sin(ang)], 1).tolist() + [[0.0, 10.0]]
    X = np.array(pts, np.float32)
    c = np.zeros((1, d), np.float32)
    st, vec = oracle.prune_stats(X, c, np.zeros(10, np.int32))
    assert st[0, 2] == pytest.approx(1.9, rel=1e-6)
    assert st[0, 3] == pytest.approx(2.7, rel=1e-6)
    assert st[0, 8] == pytest.approx(0.1)
    np.testing.assert_allclose(vec[0, 2], [0.0, 10.0], atol=1e-6)


@pytest.mark.parametrize("d", [4, 16])
def test_principal_axes_match_eigh_when_the_gap_is_clear(d):
    rng = np.random.default_rng(2 + d)
    scales = np.ones(d) * 0.3
    scales[1], scales[3] = 4.0, 2.0  # eigenvalues ~16 and ~4, the rest ~0.09
    rot = np.linalg.qr(rng.normal(size=(d, d)))[0]
    pts = (rng.normal(size=(400, d)) * scales) @ rot.T + 5.0
    X = pts.astype(np.float32)
    c = X.astype(np.float64).mean(0, keepdims=True).astype(np.float32)
    st, vec = oracle.prune_stats(X, c, np.zeros(400, np.int32))
    r = X.astype(np.float64) - c.astype(np.float64)
    w, V = np.linalg.eigh(r.T @ r / len(r))
    np.testing.assert_allclose(st[0, 9:11], [w[-1], w[-2]], rtol=1e-9)
    assert abs(vec[0, 0] @ V[:, -1]) == pytest.approx(1.0, abs=1e-9)
    assert abs(vec[0, 1] @ V[:, -2]) == pytest.approx(1.0, abs=1e-9)
    assert vec[0, 0] @ vec[0, 1] == pytest.approx(0.0, abs=1e-9)


def _hand_index():
    # list 0 around (0, 0): (+-3, 0), (0, +-1); list 1 around (10, 0): (10 +- 1, 0), (10, +-2)
    X = np.array([[3, 0], [-3, 0], [0, 1], [0, -1], [11, 0], [9, 0], [10, 2], [10, -2]], np.float32)
    assign = np.array([0, 0, 0, 0, 1, 1, 1, 1], np.int32)
    c = np.array([[0, 0], [10, 0]], np.float32)
    return X, assign, c


def test_hand_example_stats():
    X, assign, c = _hand_index()
    st, vec = oracle.prune_stats(X, c, assign)
    # list 0: distances 3, 3, 1, 1; second moment diag(4.5, 0.5)
    np.testing.assert_allclose(st[0], [4, 3, 2, 1, 0, 0.5, 0, 0.5, 0, 4.5, 0.5, 0], atol=1e-12)
    assert abs(vec[0, 0, 0]) == pytest.approx(1.0) and abs(vec[0, 1, 1]) == pytest.approx(1.0)
    # list 1: distances 1, 1, 2, 2; second moment diag(0.5, 2)
    np.testing.assert_allclose(st[1], [4, 2, 1.5, 0.5, 0, 0.5, 0, 0.5, 0, 2, 0.5, 0], atol=1e-12)
    assert abs(vec[1, 0, 1]) == pytest.approx(1.0) and abs(vec[1, 1, 0]) == pytest.approx(1.0)


def test_hand_example_features_closed_form():
    X, assign, c = _hand_index()
    st, vec = oracle.prune_stats(X, c, assign)
    Q = np.array([[0, 4]], np.float32)
    f = oracle.prune_features(Q, c, np.array([[0, 1]], np.int32), st, vec)[0]
    s = math.sqrt(116.0)  # |(0, 4) - (10, 0)|
    # nearest probe: D = D0 = 4, u = (0, 1), rho 3, mu 2, sigma 1
    want0 = [4 / 3, 1, 0.25, math.log(5), 0.75, 0.5, 0.25, 0, 0.5, 0, 0.5, 0,
             0.0, 0.5 / 16, 0, 4 / 3]
    # second probe: u = (-10, 4) / s; v1 = e1 (lambda 2), v2 = e0 (lambda 0.5)
    want1 = [s / 2, s / 4, (s - 2) / 4, math.log(5), 0.5, 1.5 / 4, 0.5 / 4, 0, 0.5, 0, 0.5, 0,
             2 * (16 / 116) / 16, 0.5 * (100 / 116) / 16, 0, 4 / 3]
    np.testing.assert_allclose(f[0], want0, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(f[1], want1, rtol=1e-9, atol=1e-12)
    # rows beyond the query's nprobe are zero
    f1 = oracle.prune_features(Q, c, np.array([[0, 1]], np.int32), st, vec, nprobe=np.array([1]))[0]
    np.testing.assert_allclose(f1[0], want0, rtol=1e-9, atol=1e-12)
    assert not f1[1].any()


def test_prune_prob_matches_torch_layers():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    F, H = oracle.PRUNE_NFEAT, oracle.PRUNE_H
    w = rng.normal(size=oracle.mlp_nparams(F, H, H)) * 0.3
    feats = rng.normal(size=(7, 3, F)) * 2 + 1
    mu, sd = rng.normal(size=F), rng.uniform(0.5, 2.0, size=F)
    got = oracle.prune_prob(feats, mu, sd, w)
    o = 0
    W1 = w[o:o + H * F].reshape(H, F); o += H * F
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = w[o:o + 2]
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    x = (t(feats.reshape(-1, F)) - t(mu)) / t(sd)
    h = torch.relu(torch.nn.functional.linear(x, t(W1), t(b1)))
    h = torch.relu(torch.nn.functional.linear(h, t(W2), t(b2)))
    p = torch.sigmoid(torch.nn.functional.linear(h, t(W3), t(b3)))[:, 0]
    np.testing.assert_allclose(got.reshape(-1), p.numpy(), rtol=1e-12)


def test_prune_keep_invariants():
    rng = np.random.default_rng(6)
    prob = rng.uniform(size=(50, 9))
    npb = rng.integers(1, 10, size=50)
    keep = oracle.prune_keep(prob, 0.4, nprobe=npb)
    for q, k in enumerate(keep):
        assert k[0] == 0 and k == sorted(k) and all(r < npb[q] for r in k)
        for r in range(npb[q]):
            if r > 0:
                assert (r in k) == (prob[q, r] > 0.4)
    # theta >= 1 keeps only the nearest probe, theta < 0 keeps every probe
    assert all(k == [0] for k in oracle.prune_keep(prob, 1.0, P=9))
    assert all(k == list(range(9)) for k in oracle.prune_keep(prob, -1.0, P=9))


def test_prune_labels_hand_example():
    assign = np.array([0, 0, 1, 2, 2, 3], np.int32)
    probes = np.array([[2, 0, 1, 3]], np.int32)
    ids = np.array([[4, 0, 5]])
    dists = np.array([[1.0, 2.0, 3.5]])
    # true k-th distance 2.0: ids 4 (list 2) and 0 (list 0) are true neighbours, 5 is not
    y = oracle.prune_labels(ids, dists, np.array([2.0]), assign, probes, P=4)
    np.testing.assert_array_equal(y, [[1, 1, 0, 0]])
    # inner product: larger is better
    y = oracle.prune_labels(ids, -dists, np.array([-2.0]), assign, probes, P=4, ip=True)
    np.testing.assert_array_equal(y, [[1, 1, 0, 0]])
    # only the first P ranks are labelled
    y = oracle.prune_labels(ids, dists, np.array([2.0]), assign, probes, P=1)
    np.testing.assert_array_equal(y, [[1, 0, 0, 0]])
