"""Pins of the component-filtration oracle (Sec. 4.3, Alg. 1 / Alg. 2).

The per-dimension fraction (values that are 0 or within one standard
deviation of the mean) is checked on dimensions whose answer is known in
closed form, the moments against numpy, and the keep / padding rules on hand
cases.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth


def test_fraction_closed_forms():
    rng = np.random.default_rng(0)
    n = 20000
    two = np.where(np.arange(n) < 0.7 * n, 3.0, 8.0)  # value 3 with p = 0.7, 8 with 0.3
    X = np.stack([
        np.full(n, 5.0),                      # constant: every value is the mean
        np.zeros(n),                          # all zero
        np.where(np.arange(n) % 2, 1.0, -1.0),  # +-1: mean 0, std 1, all within one std
        two,                                  # two values: only the majority is within one std
        rng.normal(2.0, 3.0, size=n),         # Gaussian: P(|x - mu| <= sigma) = erf(1 / sqrt 2)
        np.where(rng.uniform(size=n) < 0.9, 0.0, rng.uniform(50, 60, size=n)),  # zero 90%
    ], axis=1).astype(np.float32)
    mu, sd, fr = oracle.component_stats(X)
    np.testing.assert_allclose(mu, X.astype(np.float64).mean(0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sd, X.astype(np.float64).std(0), rtol=1e-12, atol=1e-12)
    assert fr[0] == 1.0 and fr[1] == 1.0 and fr[2] == 1.0
    # p = 0.7: |3 - mu| = 0.3 |a - b| <= sigma = |a - b| sqrt(0.21); |8 - mu| = 0.7 |a - b| > sigma
    assert fr[3] == pytest.approx(0.7, abs=1e-12)
    assert fr[4] == pytest.approx(math.erf(1 / math.sqrt(2)), abs=0.01)
    assert fr[5] >= 0.9 - 0.01  # the zeros count whatever the spread of the rest


def test_keep_and_padding_rules():
    frac = np.array([0.5, 0.99, 1.0, 0.2, 0.995, 0.7])
    np.testing.assert_array_equal(oracle.component_keep(frac, 0.99), [0, 1, 3, 5])
    np.testing.assert_array_equal(oracle.component_dims([0, 1, 3, 5], 3), [0, 1, 3, 5, -1, -1])
    np.testing.assert_array_equal(oracle.component_dims([0, 1, 3, 5], 2), [0, 1, 3, 5])
    A = np.arange(12, dtype=np.float32).reshape(2, 6)
    np.testing.assert_array_equal(oracle.filter_rows(A, np.array([5, 0, -1])), [[5, 0, 0], [11, 6, 0]])


def test_image_like_workload_drops_its_background():
    X = synth.base(6, n=6000)
    _, _, fr = oracle.component_stats(X)
    keep = oracle.component_keep(fr, 0.99)
    img = np.zeros((28, 28), bool)
    img[2:26, 2:26] = True
    np.testing.assert_array_equal(keep, np.nonzero(img.reshape(-1))[0])
