"""Pins of the oracle's Philox4x32-10 and of its uniform variates."""
import os

import numpy as np
import pytest

import oracle
from tests import fp64_paths


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(oracle.philox4x32_10(ctr, key)) == want
        assert fp64_paths.philox_py(ctr, key) == want


def test_counter_and_key_sensitivity():
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert oracle.philox4x32_10(c, [5, 6]) != base
    assert oracle.philox4x32_10([1, 2, 3, 4], [5, 7]) != base


def test_uniforms_range_mean_variance():
    # 20000 draws of 2 uniforms; exact range [-1, 1), mean 0, variance 1/3.
    xs = []
    for cell in range(100):
        xs.append(oracle.draws(cell * 7919, 3, 200, seed=12345))
    xs = np.concatenate(xs).ravel().astype(np.float64)
    assert xs.min() >= -1.0 and xs.max() < 1.0
    n = xs.size
    assert abs(xs.mean()) < 4 * np.sqrt(1 / 3 / n)
    assert abs(xs.var() - 1 / 3) < 4 * np.sqrt(4 / 45 / n)
    hist, _ = np.histogram(xs, bins=32, range=(-1, 1))
    expct = n / 32
    chi2 = ((hist - expct) ** 2 / expct).sum()
    assert chi2 < 70  # 31 dof, p ~ 1e-4


def test_uniforms_quantised_to_2_pow_minus_23():
    xs = oracle.draws(17, 0, 64, seed=1).ravel().astype(np.float64)
    k = (xs + 1.0) * 2.0 ** 23
    assert np.all(k == np.round(k))


def test_draws_match_independent_python():
    for n in range(10):
        a = oracle.draw(123, 45, n, seed=(7 << 32) | 9)
        b = fp64_paths.uniforms(123, 45, n, (7 << 32) | 9)
        assert float(a[0]) == b[0] and float(a[1]) == b[1]


def test_even_and_odd_moves_use_distinct_words():
    xs = oracle.draws(5, 6, 400, seed=0).astype(np.float64)
    even, odd = xs[0::2], xs[1::2]
    assert not np.any(np.all(even == odd, axis=1))
    c = np.corrcoef(even[:, 0], odd[:, 0])[0, 1]
    assert abs(c) < 0.25
