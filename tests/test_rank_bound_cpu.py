"""The list ranking's bound on its 16-bit scores, pinned on the CPU.

The ranking re-scores in FP32 every list whose given (tensor-core) score is
within 2 err of the P-th, so err must bound |given - exact| for every list.
This restates the bound -- for 16-bit operands (FP16 when every centroid
element is below 2^14, else BF16):
  e = (rel |q| max|c| + sub) 1.0001,  rel = (2u + u^2) + d 4.8e-7,
  sub = 2^-25 sqrt(d) (|q| + max|c|) 1.01 for FP16 (subnormal elements), 0 for BF16,
  err = (2 e for L2, e for spherical) + (d + 8) 1.2e-7 (|q| + max|c|)^2
-- and checks it against scores evaluated as the kernel does (operands
rounded to 16 bits, the dot product summed in FP32 in two orders, L2 as
FP32 ||c||^2 - 2 dot by one FMA) on random and adversarial data: tiny
magnitudes (FP16 subnormals), wide dynamic range, rows near the FP16 limit,
and rows whose every element rounds up by nearly u with the query aligned
(FP16 and BF16), which come within a few percent of the bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def r16(x, fp16):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return (t.to(torch.float16) if fp16 else t.to(torch.bfloat16)).to(torch.float32).numpy()


def dot_f32(a, b, pairwise):
    t = (a * b).astype(np.float32)
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


def bound(qn, cmax, d, fp16, spherical, mistake=None):
    u2 = 9.77e-4 + 1e-6 if fp16 else 0.0078125 + 6.2e-5
    if mistake == "u halved":
        u2 /= 2
    rel = u2 + d * 4.8e-7
    sub = 2.0 ** -25 * np.sqrt(d) * (qn + cmax) * 1.01 if fp16 and mistake != "no subnormal term" else 0.0
    e = (rel * qn * cmax + sub) * 1.0001
    r = (d + 8) * 1.2e-7 * (qn + cmax) ** 2
    return (e if spherical else 2 * e) + r


def data(rng, kind, d, L):
    if kind == "normal":
        return rng.normal(size=(L, d)), rng.normal(size=d)
    if kind == "tiny":  # FP16 subnormals throughout
        return rng.normal(size=(L, d)) * 1e-6, rng.normal(size=d) * 1e-6
    if kind == "range":  # magnitudes over ten decades
        return rng.normal(size=(L, d)) * 10.0 ** rng.uniform(-8, 2, size=(L, d)), \
            rng.normal(size=d) * 10.0 ** rng.uniform(-8, 2, size=d)
    if kind == "big":  # centroids near the FP16 limit (BF16 then)
        return rng.uniform(-2e4, 2e4, size=(L, d)), rng.uniform(-1e3, 1e3, size=d)
    if kind in ("aligned", "aligned_bf16"):
        # every element just above a halfway point, so it rounds up by nearly
        # u (FP16: 1 + 2^-11 + 2^-20 -> 1 + 2^-10; BF16: 1 + 2^-8 + 2^-16 ->
        # 1 + 2^-7), and the query aligned with row 0, the largest row: the
        # operand term 2u + u^2 is nearly attained
        m, scale = (1 + 2.0 ** -11 + 2.0 ** -20, 1.0) if kind == "aligned" else (1 + 2.0 ** -8 + 2.0 ** -16, 2.0 ** 15)
        C = rng.choice([-1.0, 1.0], size=(L, d)) * m * scale * 2.0 ** rng.integers(-4, 1, size=(L, 1))
        C[0] = np.sign(C[0]) * m * scale
        return C, np.sign(C[0]) * m * scale  # |q| = |c_0|: the norm term stays small beside it
    raise ValueError(kind)


def worst_ratio(kind, spherical, mistake=None):
    """Largest |given - exact| / err over 20 draws and two summation orders;
    also whether FP16 operands were used."""
    rng = np.random.default_rng(hash((kind, spherical)) % 2 ** 32)
    d, L = 96, 64
    worst, fp16 = 0.0, None
    for _ in range(20):
        C, q = data(rng, kind, d, L)
        C = C.astype(np.float32)
        q = q.astype(np.float32)
        fp16 = np.abs(C).max() < 16384.0
        if fp16 and np.abs(q).max() > 6.0e4:
            continue  # the kernel gives no bound then (every list re-scored)
        cn = (C.astype(np.float64) ** 2).sum(1)
        cmax = np.float32(np.sqrt(np.float32(cn.max())))
        qn = float(np.sqrt(np.float32((q.astype(np.float64) ** 2).sum())))
        err = bound(qn, float(cmax), d, fp16, spherical, mistake)
        qt, Ct = r16(q, fp16), r16(C, fp16)
        exact = -(C.astype(np.float64) @ q) if spherical else cn - 2.0 * (C.astype(np.float64) @ q)
        for pw in (False, True):
            dot = np.array([dot_f32(Ct[i], qt, pw) for i in range(L)], dtype=np.float32)
            if spherical:
                given = -dot
            else:
                given = np.array([np.float32(np.float32(-2.0) * dot[i] + np.float32(cn[i])) for i in range(L)])
            worst = max(worst, float(np.abs(given.astype(np.float64) - exact).max() / err))
    return worst, fp16


@pytest.mark.parametrize("kind", ["normal", "tiny", "range", "big", "aligned", "aligned_bf16"])
@pytest.mark.parametrize("spherical", [False, True])
def test_16bit_score_bound_holds(kind, spherical):
    worst, fp16 = worst_ratio(kind, spherical)
    assert worst <= 1.0, (kind, fp16, worst)
    if kind.startswith("aligned"):  # the operand term nearly attained
        assert fp16 == (kind == "aligned")
        assert worst > 0.75, worst


@pytest.mark.parametrize("mistake,kind", [("u halved", "aligned"), ("u halved", "aligned_bf16"),
                                          ("no subnormal term", "tiny")])
def test_16bit_pin_catches_a_smaller_bound(mistake, kind):
    """The same check with a plausible mistake planted in the restated bound
    (the unit roundoff of FP16 or BF16 halved, FP16's subnormal term left
    out) fails on the rows built for it."""
    assert worst_ratio(kind, True, mistake)[0] > 1.0
