"""The exact re-rank's band selection, restated on the CPU.

The band reads a low-precision copy of each candidate row, bounds the FP32
distance from it (|d~ - d| <= e), takes U = the k-th smallest d~ + e and
re-reads in FP32 only the candidates with d~ - e <= U; the k best of those
are the k best of all.  This restates that rule on the oracle's candidates
of a small index and checks that the FP32 top k always survives, with the
two passes' own summation orders: the FP32 pass with lane l holding
coordinates 4l .. 4l + 3 and a tree over lane bits 4 .. 0, the band pass with
8 lanes per row (chunks j, j + 8, j + 16, j + 24 in FP32 pairs, then a tree
over the 8 lanes).  Rows: a byte-valued set (U8 copies, exact: r = 0, the
band is the evaluation term alone) and the real-valued set (BF16 copies,
r = |x~ - x| per row).  Bound (L2): e = (2 r s + r^2 + g (s^2 + (s + r)^2))
(1 + 2^-10), s = sqrt(d~ (1 + 2 g)) (1 + 2^-20), g = 2^-20.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2511_03298_gb300 import synth  # noqa: E402

F32 = np.float32
G, SAFE = 2.0 ** -20, 1.0 + 2.0 ** -10


def fma(a, b, c):
    """a b + c rounded to FP32 (the product is exact in FP64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def fp32_pass(q, rows):
    """Squared distances in the FP32 pass's order (d = 128)."""
    e = (q[None, :] - rows).astype(F32).reshape(len(rows), 32, 4)
    a = fma(e[:, :, 0], e[:, :, 0], fma(e[:, :, 1], e[:, :, 1],
                                          fma(e[:, :, 2], e[:, :, 2], (e[:, :, 3] * e[:, :, 3]).astype(F32))))
    while a.shape[1] > 1:  # lane bit 4 first, then 3, 2, 1, 0
        h = a.shape[1] // 2
        a = (a[:, :h] + a[:, h:]).astype(F32)
    return a[:, 0]


def band_pass(q, rows):
    """Squared distances in the band pass's order: 8 lanes per row."""
    d = rows.shape[1]
    e = (q[None, :] - rows).astype(F32)
    lanes = []
    for j in range(8):
        ax = np.zeros(len(rows), F32)
        ay = np.zeros(len(rows), F32)
        for k in range(4):
            c = j + 8 * k
            if 4 * c >= d:
                continue
            ax = fma(e[:, 4 * c], e[:, 4 * c], ax)
            ay = fma(e[:, 4 * c + 1], e[:, 4 * c + 1], ay)
            ax = fma(e[:, 4 * c + 2], e[:, 4 * c + 2], ax)
            ay = fma(e[:, 4 * c + 3], e[:, 4 * c + 3], ay)
        lanes.append((ax + ay).astype(F32))
    p = [(lanes[j] + lanes[j + 4]).astype(F32) for j in range(4)]
    return ((p[0] + p[2]).astype(F32) + (p[1] + p[3]).astype(F32)).astype(F32)


def bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def row_errors(X, Xc):
    """|x~ - x| per row from FP64 sums, rounded up to FP32 (0 when exact)."""
    r2 = ((X.astype(np.float64) - Xc.astype(np.float64)) ** 2).sum(1)
    r = np.sqrt(r2) * (1 + 2.0 ** -40)
    return np.where(r2 == 0, 0.0, np.nextafter(r.astype(F32), F32(np.inf)).astype(np.float64))


@pytest.fixture(scope="module")
def index():
    X = synth.base(1)
    Q = synth.queries(1)[:60]
    ix = oracle.build_index(X, 64, 64, False, synth.build_perm(1, len(X)), iters=6)
    return ix, Q


def byte_valued(ix, Q):
    """The same index mapped onto integer coordinates in [0, 255] (rows,
    centroids and codebooks together, so the codes still encode the rows)."""
    X = np.clip(np.rint(12.0 * np.asarray(ix["X"], np.float64) + 128.0), 0, 255).astype(F32)
    out = dict(ix, X=X, c_rank=(12.0 * np.asarray(ix["c_rank"], np.float64) + 128.0).astype(F32),
               c_mean=(12.0 * np.asarray(ix["c_mean"], np.float64) + 128.0).astype(F32),
               codebook=(12.0 * np.asarray(ix["codebook"], np.float64)).astype(F32))
    return out, (12.0 * np.asarray(Q, np.float64) + 128.0).astype(F32)


@pytest.mark.parametrize("rows", ["u8", "bf16"])
def test_band_keeps_the_fp32_top_k(index, rows):
    ix, Q = index
    if rows == "u8":
        ix, Q = byte_valued(ix, Q)
        X = ix["X"]
        Xc = X.copy()  # a byte holds every coordinate
    else:
        X = np.asarray(ix["X"], F32)
        Xc = bf16(X)
    r_all = row_errors(X, Xc)
    if rows == "u8":
        assert np.all(r_all == 0.0)
    else:
        assert np.all(r_all > 0.0)
    survivors = []
    for k, R in ((10, 100), (32, 200), (1, 40)):
        for qi in range(len(Q)):
            q = Q[qi].astype(F32)
            probes = oracle.rank(Q[qi], ix["c_rank"], False, 9)[0]
            Ql, bias, _ = oracle.lut_q8(Q[qi], ix, probes)
            keys = np.asarray(oracle.scan_topr(ix, probes, Ql, bias, R), np.uint64)
            ids = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
            d32 = fp32_pass(q, X[ids])
            dt = band_pass(q, Xc[ids]).astype(np.float64)
            r = r_all[ids]
            s = np.sqrt(np.maximum(dt, 0.0) * (1 + 2 * G)) * (1 + 2.0 ** -20)
            e = (2 * r * s + r * r + G * (s * s + (s + r) ** 2)) * SAFE
            lo, hi = dt - e, dt + e
            U = np.sort(hi)[k - 1]
            keep = lo <= U
            best = np.lexsort((ids, d32))[:k]  # the FP32 top k by (distance, id)
            assert keep[best].all(), (rows, k, R, qi)
            survivors.append(keep.sum() / k)
    # the exact rows' band holds little more than the k best and their ties
    if rows == "u8":
        assert np.mean(survivors) < 2.0, np.mean(survivors)
