"""The exact re-rank's band: the bound on |d~ - d| it relies on.

The re-rank may skip a candidate's FP32 distance d when a distance d~
computed in FP32 from the BF16-rounded row, widened by a bound e, already
places the candidate above k others.  This checks the bound's derivation on
the CPU, independently of the kernel: for random and adversarial rows (large
norms, near-duplicates of the query, wide dynamic range, integer rows that
BF16 holds exactly, inner products), |d~ - d| <= e, with d and d~ evaluated
in FP32 in three orders (sequential, pairwise, and the BF16 pass's: 8 lanes
of 4-coordinate chunks in FP32 pairs, then a tree over the lanes), and e
built from the same terms and constants:
  L2: e = (2 r s + r^2 + g (s^2 + (s + r)^2)) (1 + 2^-10),
      s = sqrt(d~ (1 + 2 g)) (1 + 2^-20)
  IP: e = |q| (r + 2.01 g (n + r)) (1 + 2^-10), |q| taken with (1 + 2^-18)
n >= |x| and r >= |x~ - x| (the row's own BF16 rounding error), g = 2^-20.
The worst case of r is 2^-8 n (BF16 keeps 8 significant bits), which the
rows here also check.
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


def fma32(a, b, c):
    """a b + c rounded to FP32 (the product is exact in FP64)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def lanes8_sum(u, v):
    """Sum over t of u_t v_t in the BF16 pass's order: lane j takes chunks
    j, j + 8, j + 16, j + 24 (coordinates 4c .. 4c + 3) into two FP32
    accumulators (even and odd coordinates), adds them, and the 8 lane sums
    go through the tree ((0 + 4) + (2 + 6)) + ((1 + 5) + (3 + 7))."""
    d = len(u)
    a = []
    for j in range(8):
        ax = ay = np.float32(0)
        for k in range(4):
            c = j + 8 * k
            if 4 * c >= d:
                continue
            ax = fma32(u[4 * c], v[4 * c], ax)
            ay = fma32(u[4 * c + 1], v[4 * c + 1], ay)
            ax = fma32(u[4 * c + 2], v[4 * c + 2], ax)
            ay = fma32(u[4 * c + 3], v[4 * c + 3], ay)
        a.append(np.float32(ax + ay))
    p = [np.float32(a[j] + a[j + 4]) for j in range(4)]
    return np.float32(np.float32(p[0] + p[2]) + np.float32(p[1] + p[3]))


ORDERS = ("seq", "pairwise", "lanes8")


def l2_f32(q, x, order):
    e = (q - x).astype(np.float32)
    if order == "lanes8":
        return lanes8_sum(e, e)
    return f32_sum((e * e).astype(np.float32), order == "pairwise")


def ip_f32(q, x, order):
    if order == "lanes8":
        return -lanes8_sum(q, x)
    return -f32_sum((q * x).astype(np.float32), order == "pairwise")


def row_bounds(x, xb):
    """(n, r): |x| and |x~ - x| from FP64 sums, rounded up to FP32."""
    n = np.sqrt((x.astype(np.float64) ** 2).sum()) * (1 + 2.0 ** -40)
    r2 = ((x.astype(np.float64) - xb.astype(np.float64)) ** 2).sum()
    r = 0.0 if r2 == 0 else np.sqrt(r2) * (1 + 2.0 ** -40)
    return float(np.nextafter(np.float32(n), np.float32(np.inf))), \
        float(np.nextafter(np.float32(r), np.float32(np.inf))) if r > 0 else 0.0


def bound_l2(dt, r, mistake=None):
    sq = np.sqrt(max(float(dt), 0.0) * (1 + 2 * G)) * (1 + 2.0 ** -20)
    two = 1.0 if mistake == "r s in place of 2 r s" else 2.0
    return (two * r * sq + r * r + G * (sq * sq + (sq + r) ** 2)) * SAFE


def bound_ip(qn, n, r, mistake=None):
    rr = r / 2 if mistake == "r / 2 for inner products" else r
    return qn * (1 + 2.0 ** -18) * (rr + 2.01 * G * (n + r)) * SAFE


def cases(rng, d):
    yield rng.normal(size=d), rng.normal(size=d)                      # generic
    q = rng.normal(size=d) * 300
    yield q, q + rng.normal(size=d) * 1e-3                             # near-duplicate, large norm
    yield rng.uniform(0, 255, size=d), rng.uniform(0, 255, size=d)     # SIFT-like magnitudes
    x = rng.normal(size=d) * np.exp(rng.uniform(-20, 20, size=d))      # wide dynamic range
    yield rng.normal(size=d), x
    yield np.zeros(d), rng.normal(size=d)                              # zero query
    yield rng.uniform(0, 255, size=d), np.rint(rng.uniform(0, 255, size=d))  # integer row: r = 0
    x = np.rint(rng.uniform(0, 255, size=d))
    yield x + rng.normal(size=d) * 0.01, x                             # integer row, query close by
    # queries along the row's own rounding error, where Cauchy-Schwarz is tight:
    # <q, x~ - x> = |q| r (inner products), q - x~ parallel to x~ - x (L2)
    x = rng.normal(size=d).astype(np.float32)
    dx = bf16(x).astype(np.float64) - x
    u = dx / np.linalg.norm(dx)
    yield 3.0 * u, x
    yield bf16(x) + 5.0 * u, x


def worst_ratios(d, mistake=None, draws=60):
    """Largest |d~ - d| / e for L2 and for inner products over the cases,
    nine pairs of summation orders each."""
    rng = np.random.default_rng(d)
    wl = wi = 0.0
    for _ in range(draws):
        for q, x in cases(rng, d):
            q = q.astype(np.float32)
            x = x.astype(np.float32)
            xb = bf16(x)
            n, r = row_bounds(x, xb)
            assert r <= EPS * n * (1 + 2.0 ** -20) + 1e-37  # the format's worst case
            if np.all(x == np.rint(x)) and np.abs(x).max() <= 256:
                assert r == 0.0  # BF16 holds integers up to 256 exactly
            qn = float(np.sqrt((q.astype(np.float64) ** 2).sum()))
            for o_exact in ORDERS:
                d32 = float(l2_f32(q, x, o_exact))
                i32 = float(ip_f32(q, x, o_exact))
                for o_bf in ORDERS:
                    db = float(l2_f32(q, xb, o_bf))
                    e = bound_l2(db, r, mistake)
                    dev = abs(db - d32)
                    wl = max(wl, dev / e if e > 0 else (0.0 if dev == 0 else np.inf))
                    ib = float(ip_f32(q, xb, o_bf))
                    ei = bound_ip(qn, n, r, mistake)
                    dev = abs(ib - i32)
                    wi = max(wi, dev / ei if ei > 0 else (0.0 if dev == 0 else np.inf))
    return wl, wi


@pytest.mark.parametrize("d", [16, 100, 128])
def test_band_bound_holds(d):
    wl, wi = worst_ratios(d)
    assert wl < 1.0 and wi <= 1.0, (d, wl, wi)


@pytest.mark.parametrize("mistake", ["r s in place of 2 r s", "r / 2 for inner products"])
def test_band_pin_catches_a_smaller_bound(mistake):
    """The same check with a plausible mistake planted in the restated bound
    (the cross term's factor 2 dropped, half the row's error for inner
    products) fails on the rows above."""
    wl, wi = worst_ratios(128, mistake)
    assert (wl if mistake.startswith("r s") else wi) > 1.0, (mistake, wl, wi)


def test_integer_rows_band_is_the_evaluation_term():
    """For rows BF16 holds exactly (r = 0) the band is the FP32 evaluation
    term alone, which still covers two evaluation orders; on SIFT-like
    integer rows at a nearest neighbour's distance (about 5e4) the band is
    below one unit of the distance, so it keeps hardly more than the ties
    with the k-th."""
    rng = np.random.default_rng(11)
    for _ in range(100):
        x = np.rint(rng.uniform(0, 255, size=128)).astype(np.float32)
        q = (x + np.rint(rng.normal(size=128) * 20)).astype(np.float32)
        n, r = row_bounds(x, bf16(x))
        assert r == 0.0
        d_a, d_b = float(l2_f32(q, x, "seq")), float(l2_f32(q, x, "lanes8"))
        e = bound_l2(d_b, 0.0)
        assert abs(d_a - d_b) <= e < 1.0


def test_bound_is_tight_enough_to_prune():
    """On SIFT-like rows the band is a small fraction of the distance gaps it
    must resolve: for the 10 nearest of 200 candidates, the BF16 lower bound
    of the 200th exceeds the 10th's upper bound (the pruning can happen)."""
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 255, size=(200, 128)).astype(np.float32)
    q = X[0] + rng.normal(size=128).astype(np.float32) * 10
    Xb = bf16(X)
    rb = [row_bounds(x, xb)[1] for x, xb in zip(X, Xb)]
    db = np.array([float(l2_f32(q, xb, "pairwise")) for xb in Xb])
    e = np.array([bound_l2(v, ri) for v, ri in zip(db, rb)])
    U = np.sort(db + e)[9]
    assert (db - e > U).sum() > 100
