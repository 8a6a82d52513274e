"""The list ranking's bound on its FP8 scores, pinned on the CPU.

With the FP8 option every query and centroid row is scaled by a power of two
s = 2^(e - 8), e the exponent of the row's largest magnitude (m 2^e, m in
[0.5, 1)), and rounded to e4m3; the dot product of the rounded rows is summed
and multiplied by s_q s_c.  The ranking re-scores in FP32 every list within 2
err of the P-th given score, so err must bound |given - exact|.  This
restates the bound:
  rel = (2u + u^2) + 2 (1 + u) 2^-10 sqrt(d) / 128 + d 2^-13 (1 + u)^2 + 1e-6,
  u = 2^-4 (e4m3 keeps 4 significant bits; 2^-10 is half its subnormal spacing),
  e = rel |q| max|c| 1.0001,
  err = (2 e for L2, e for spherical) + (d + 8) 1.2e-7 (|q| + max|c|)^2
and checks it against scores evaluated with the e4m3 rounding, the exact
rescaling and three accumulations of the products: FP32 in order, FP32
pairwise, and a 13-significant-bit accumulator (the bound's assumption on
the tensor core's accumulation).  Data: normal rows, magnitudes over ten
decades within a row and rows of one large element among small ones (most
elements then in e4m3's subnormal range or flushed to zero), and rows whose
every element rounds up by nearly u with the query aligned to one of them,
which comes within 0.82 of the bound (u = 2^-5, or 2u replaced by u, fails).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not hasattr(torch, "float8_e4m3fn"):
    pytest.skip("this PyTorch has no e4m3 type", allow_module_level=True)

U = 2.0 ** -4


def row_scale(x):
    """2^(e - 8) for a row whose largest magnitude is m 2^e, m in [0.5, 1)."""
    mx = np.abs(x).max(axis=-1)
    _, e = np.frexp(mx)
    return np.where(mx > 0, np.ldexp(1.0, e - 8), 1.0).astype(np.float32)


def e4m3(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.float8_e4m3fn).to(torch.float32).numpy()


def round_bits(x, p):
    """x rounded to nearest with p significant bits (ties away; float64)."""
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 2.0 ** p) / 2.0 ** p, e)


def dots(Cq, qq, mode):
    """Sum over t of Cq[:, t] * qq[t] for every row; the products are exact."""
    prod = Cq.astype(np.float64) * qq.astype(np.float64)[None, :]
    if mode == "pairwise":
        t = prod.astype(np.float32)
        while t.shape[1] > 1:
            if t.shape[1] % 2:
                t = np.concatenate([t, np.zeros((t.shape[0], 1), np.float32)], axis=1)
            t = (t[:, 0::2] + t[:, 1::2]).astype(np.float32)
        return t[:, 0]
    acc = np.zeros(prod.shape[0], np.float64)
    for j in range(prod.shape[1]):
        acc = acc + prod[:, j]
        acc = acc.astype(np.float32).astype(np.float64) if mode == "seq" else round_bits(acc, 13)
    return acc.astype(np.float32)


def fp8_rel(d, u=U, two=2.0):
    return (two * u + u * u) + 2 * (1 + u) * 2.0 ** -10 * np.sqrt(d) / 128 + d * 2.0 ** -13 * (1 + u) ** 2 + 1e-6


def bound(qn, cmax, d, spherical, rel=fp8_rel):
    e = rel(d) * qn * cmax * 1.0001
    r = (d + 8) * 1.2e-7 * (qn + cmax) ** 2
    return (e if spherical else 2 * e) + r


def data(rng, kind, d, L):
    if kind == "normal":
        return rng.normal(size=(L, d)), rng.normal(size=d)
    if kind == "range":  # magnitudes over ten decades
        return rng.normal(size=(L, d)) * 10.0 ** rng.uniform(-8, 2, size=(L, d)), \
            rng.normal(size=d) * 10.0 ** rng.uniform(-8, 2, size=d)
    if kind == "spike":  # one large element per row, the rest near e4m3's subnormal range
        C = rng.normal(size=(L, d)) * 0.02
        C[np.arange(L), rng.integers(0, d, size=L)] = rng.choice([-1.0, 1.0], size=L) * 40.0
        q = rng.normal(size=d) * 0.02
        q[rng.integers(0, d)] = 30.0
        return C, q
    if kind == "aligned":  # every element rounds up by nearly u, q aligned with row 0
        # magnitude 2^k 0.5313: scaled to 136.01, just above the halfway point 136 of
        # [128, 144], so it rounds to 144 (relative error 0.0587, nearly 2^-4)
        C = rng.choice([-1.0, 1.0], size=(L, d)) * 0.5313 * 2.0 ** rng.integers(-3, 4, size=(L, 1))
        C[0] = np.sign(C[0]) * 0.5313 * 8.0  # row 0 has the largest norm
        q = np.sign(C[0]) * 0.5313 * 4.0
        return C, q
    raise ValueError(kind)


def test_e4m3_rounding_is_the_format():
    """The rounding used below keeps 4 significant bits, has subnormal spacing 2^-9 and is
    round-to-nearest-even: checked on values whose rounding the format fixes."""
    assert e4m3(np.float32(1.0 + 2.0 ** -4)) == 1.0  # halfway: to even
    assert e4m3(np.float32(1.0 + 3 * 2.0 ** -4)) == 1.25  # halfway: to even (up)
    assert e4m3(np.float32(2.0 ** -9)) == 2.0 ** -9  # smallest subnormal
    assert e4m3(np.float32(2.0 ** -10 * 1.01)) == 2.0 ** -9
    assert e4m3(np.float32(3 * 2.0 ** -10)) == 2 * 2.0 ** -9  # halfway between 1 and 2 spacings: even
    assert e4m3(np.float32(448.0)) == 448.0
    x = np.random.default_rng(0).uniform(-255, 255, size=4096).astype(np.float32)
    y = e4m3(x)
    big = np.abs(x) >= 2.0 ** -6
    assert np.all(np.abs(y - x)[big] <= U * np.abs(x)[big])
    assert np.all(np.abs(y - x)[~big] <= 2.0 ** -10)


def test_row_scale_peaks_in_128_256():
    x = np.random.default_rng(1).normal(size=(64, 96)) * 10.0 ** np.random.default_rng(2).uniform(-6, 6, size=(64, 1))
    s = row_scale(x.astype(np.float32))
    peak = np.abs(x.astype(np.float32)).max(1) / s
    assert np.all((peak >= 128) & (peak < 256))


def worst_ratio(kind, spherical, rel=fp8_rel):
    """Largest |given - exact| / err over 20 draws and three accumulations."""
    rng = np.random.default_rng(hash(("fp8", kind, spherical)) % 2 ** 32)
    d, L = 128, 64
    worst = 0.0
    for _ in range(20):
        C, q = data(rng, kind, d, L)
        C = C.astype(np.float32)
        q = q.astype(np.float32)
        cn = (C.astype(np.float64) ** 2).sum(1)
        cmax = float(np.sqrt(np.float32(cn.max())))
        qn = float(np.sqrt(np.float32((q.astype(np.float64) ** 2).sum())))
        err = bound(qn, cmax, d, spherical, rel)
        sc, sq = row_scale(C), row_scale(q[None, :])[0]
        Cq, qq = e4m3(C / sc[:, None]), e4m3(q / sq)
        exact = -(C.astype(np.float64) @ q) if spherical else cn - 2.0 * (C.astype(np.float64) @ q)
        for mode in ("seq", "pairwise", "acc13"):
            dot = dots(Cq, qq, mode) * (sq * sc)  # powers of two: exact
            if spherical:
                given = -dot.astype(np.float64)
            else:
                given = np.array([np.float32(np.float32(-2.0) * dot[i] + np.float32(cn[i])) for i in range(L)],
                                 dtype=np.float64)
            worst = max(worst, float(np.abs(given - exact).max() / err))
    return worst


@pytest.mark.parametrize("kind", ["normal", "range", "spike", "aligned"])
@pytest.mark.parametrize("spherical", [False, True])
def test_fp8_score_bound_holds(kind, spherical):
    worst = worst_ratio(kind, spherical)
    assert worst <= 1.0, (kind, worst)
    if kind == "aligned":  # the operand rounding's term is nearly attained
        assert worst > 0.75, worst


@pytest.mark.parametrize("mistake", ["u = 2^-5", "u in place of 2u"])
def test_fp8_pin_catches_a_smaller_bound(mistake):
    """The same check with a plausible mistake planted in the restated bound
    (one bit too many for e4m3, the factor 2 of the two operands' rounding
    dropped) fails on the aligned rows."""
    rel = (lambda d: fp8_rel(d, u=2.0 ** -5)) if mistake == "u = 2^-5" else (lambda d: fp8_rel(d, two=1.0))
    assert worst_ratio("aligned", True, rel) > 1.0
