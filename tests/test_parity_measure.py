"""The parity measure of the GPU tests (tests/parity.py) on known cases: a
single row off by a relative 1e-4 of the column's largest entry fails a 1e-5
bound although the column's 2-norm error stays below it."""
import numpy as np

from parity import rel


def test_one_bad_row_fails_although_the_norm_passes():
    rng = np.random.default_rng(0)
    b = rng.normal(size=(10000, 3)) + 1j * rng.normal(size=(10000, 3))
    a = b.copy()
    a[1234, 1] += 2e-4 * np.abs(b[:, 1]).max()
    norm_only = max(np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c]) for c in range(3))
    assert norm_only < 1e-5
    assert rel(a, b) > 1e-4


def test_uniform_small_error_passes_and_shapes():
    rng = np.random.default_rng(1)
    b = rng.normal(size=(500, 2))
    a = b * (1 + 1e-7 * rng.normal(size=b.shape))
    assert rel(a, b) < 1e-6
    assert rel(a[:, 0], b[:, 0]) < 1e-6
    assert rel(b, b) == 0.0
    bad = a.copy()
    bad[3, 0] = np.nan
    assert rel(bad, b) == float("inf")
