"""The arithmetic the tensor-core scan relies on, checked on the CPU.

The scan forms each (vector, query) table sum as a product of a one-hot
expansion of the codes (FP16 1.0 entries) and the query's u8 tables stored as
FP16 1024 + T (bit pattern 0x6400 | T), accumulated in FP32.  These tests pin
(1) that bit pattern, (2) that such a product is exact for every table value
and any number of subspaces up to 128, whatever the order of the additions,
and (3) that subtracting 1024 M leaves the plain sum of Alg. 3's lookups
(the oracle's scan sums).
"""
import numpy as np

import oracle


def test_fp16_pattern_is_1024_plus_byte():
    t = np.arange(256, dtype=np.uint16)
    h = (0x6400 | t).astype(np.uint16).view(np.float16).astype(np.float64)
    np.testing.assert_array_equal(h, 1024.0 + t)
    # the byte-permute form: two table bytes -> one word of two FP16 values
    x0, x1 = 0xAB, 0x07
    word = x0 | (0x64 << 8) | (x1 << 16) | (0x64 << 24)
    pair = np.array([word], np.uint32).view(np.float16).astype(np.float64)
    np.testing.assert_array_equal(pair, [1024 + x0, 1024 + x1])


def _onehot_sums(codes, T, order):
    """FP32 accumulation of one-hot(codes) . (1024 + T) over K in `order`."""
    n, M = codes.shape
    K = 16 * M
    A = np.zeros((n, K), np.float16)
    A[np.arange(n)[:, None], 16 * np.arange(M)[None, :] + codes] = 1.0
    B = (1024 + T.reshape(-1)).astype(np.float16)
    acc = np.zeros(n, np.float32)
    for k in order:
        acc = (acc + A[:, k].astype(np.float32) * np.float32(B[k])).astype(np.float32)
    return acc


def test_one_hot_product_is_exact():
    rng = np.random.default_rng(5)
    for M in (4, 50, 64, 128):
        codes = rng.integers(0, 16, size=(64, M))
        T = rng.integers(0, 256, size=(M, 16))
        T[:, 15] = 255  # the largest entry reachable by some code
        codes[0] = 15   # a vector that sums the maximum in every subspace
        want = 1024 * M + T[np.arange(M)[None, :], codes].sum(1)
        for order in (np.arange(16 * M), rng.permutation(16 * M)):
            got = _onehot_sums(codes, T, order)
            np.testing.assert_array_equal(got.astype(np.int64), want)
        assert want.max() < 2 ** 24


def test_minus_1024M_gives_the_oracle_scan_sums():
    rng = np.random.default_rng(6)
    M = 16
    codes = rng.integers(0, 16, size=(32, M)).astype(np.uint8)
    T = rng.integers(0, 256, size=(M, 16)).astype(np.uint8)
    sums = _onehot_sums(codes.astype(np.int64), T.astype(np.int64), np.arange(16 * M)).astype(np.int64) - 1024 * M
    ref = np.array([oracle.int_dist(T, 0, codes[v]) for v in range(len(codes))])
    np.testing.assert_array_equal(sums, ref)
