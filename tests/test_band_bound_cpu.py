"""The exact re-rank's BF16 band: the bound on |d~ - d| it relies on.

The re-rank may skip a candidate's FP32 distance d when a distance d~
computed in FP32 from the BF16-rounded row, widened by a bound e, already
places the candidate above k others.  This checks the bound's derivation on
the CPU, independently of the kernel: for random and adversarial rows (large
norms, near-duplicates of the query, wide dynamic range, inner products),
|d~ - d| <= e, with d and d~ both evaluated in FP32 in two different orders
(sequential and pairwise), and e built from the same terms and constants:
  L2: e = (2 eps n s + (eps n)^2 + g (s^2 + (s + eps n)^2)) (1 + 2^-10),
      s = sqrt(d~ (1 + 2 g)) (1 + 2^-20), n >= |x|
  IP: e = |q| n (eps + 2.01 g) (1 + 2^-10), |q| taken with (1 + 2^-18)
eps = 2^-8 (BF16 round-to-nearest: 8 significant bits), g = 2^-20.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

EPS, G, SAFE = 2.0 ** -8, 2.0 ** -20, 1.0 + 2.0 ** -10


def bf16(x):
    return torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()


def f32_sum(terms, pairwise):
    """Sum of float32 terms in float32: sequentially, or as a pairwise tree."""
    t = terms.astype(np.float32)
    if not pairwise:
        acc = np.float32(0)
        for v in t:
            acc = np.float32(acc + v)
        return acc
    while len(t) > 1:
        if len(t) % 2:
            t = np.append(t, np.float32(0))
        t = (t[0::2] + t[1::2]).astype(np.float32)
    return t[0]


def l2_f32(q, x, pairwise):
    e = (q - x).astype(np.float32)
    return f32_sum((e * e).astype(np.float32), pairwise)


def ip_f32(q, x, pairwise):
    return -f32_sum((q * x).astype(np.float32), pairwise)


def bound_l2(dt, n):
    sq = np.sqrt(max(float(dt), 0.0) * (1 + 2 * G)) * (1 + 2.0 ** -20)
    en = EPS * n
    return (2 * en * sq + en * en + G * (sq * sq + (sq + en) ** 2)) * SAFE


def bound_ip(qn, n):
    return qn * (1 + 2.0 ** -18) * n * (EPS + 2.01 * G) * SAFE


def cases(rng, d):
    yield rng.normal(size=d), rng.normal(size=d)                      # generic
    q = rng.normal(size=d) * 300
    yield q, q + rng.normal(size=d) * 1e-3                             # near-duplicate, large norm
    yield rng.uniform(0, 255, size=d), rng.uniform(0, 255, size=d)     # SIFT-like magnitudes
    x = rng.normal(size=d) * np.exp(rng.uniform(-20, 20, size=d))      # wide dynamic range
    yield rng.normal(size=d), x
    yield np.zeros(d), rng.normal(size=d)                              # zero query


@pytest.mark.parametrize("d", [16, 100, 128])
def test_bf16_band_bound_holds(d):
    rng = np.random.default_rng(d)
    worst = 0.0
    for _ in range(200):
        for q, x in cases(rng, d):
            q = q.astype(np.float32)
            x = x.astype(np.float32)
            xb = bf16(x)
            n = float(np.sqrt((x.astype(np.float64) ** 2).sum()))
            for pw_exact in (False, True):
                for pw_bf in (False, True):
                    d32 = float(l2_f32(q, x, pw_exact))
                    db = float(l2_f32(q, xb, pw_bf))
                    e = bound_l2(db, n)
                    assert abs(db - d32) <= e, (d, db, d32, e)
                    worst = max(worst, abs(db - d32) / e if e > 0 else 0.0)
                    i32 = float(ip_f32(q, x, pw_exact))
                    ib = float(ip_f32(q, xb, pw_bf))
                    qn = float(np.sqrt((q.astype(np.float64) ** 2).sum()))
                    ei = bound_ip(qn, n)
                    assert abs(ib - i32) <= ei + 0.0, (d, ib, i32, ei)
    assert worst < 1.0


def test_bound_is_tight_enough_to_prune():
    """On SIFT-like rows the band is a small fraction of the distance gaps it
    must resolve: for the 10 nearest of 200 candidates, the BF16 lower bound
    of the 200th exceeds the 10th's upper bound (the pruning can happen)."""
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 255, size=(200, 128)).astype(np.float32)
    q = X[0] + rng.normal(size=128).astype(np.float32) * 10
    Xb = bf16(X)
    n = np.sqrt((X.astype(np.float64) ** 2).sum(1))
    db = np.array([float(l2_f32(q, xb, True)) for xb in Xb])
    e = np.array([bound_l2(v, ni) for v, ni in zip(db, n)])
    U = np.sort(db + e)[9]
    assert (db - e > U).sum() > 100
