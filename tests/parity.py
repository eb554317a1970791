"""Error measure of the GPU parity tests.

For each column c of a GPU result a and the oracle's b, two relative errors:
  ||a_c - b_c||_2 / ||b_c||_2           (the column as a whole)
  max_i |a_ic - b_ic| / max_i |b_ic|    (every element against the column's scale)
rel() returns the largest of them over all columns, so `rel(a, b) < tol`
bounds both: one row off by more than tol times the column's largest entry
fails even where the column norm would hide it (a ragged tile or a partition
bug touches a few rows only).  1-D inputs are one column.
"""
import numpy as np


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape:
        raise ValueError(f"shapes differ: {a.shape} vs {b.shape}")
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    worst = 0.0
    for c in range(b.shape[1]):
        d = a[:, c] - b[:, c]
        if not np.isfinite(d).all():
            return float("inf")
        nb = np.linalg.norm(b[:, c])
        mb = np.abs(b[:, c]).max() if b.shape[0] else 0.0
        nd = np.linalg.norm(d)
        md = np.abs(d).max() if d.size else 0.0
        worst = max(worst, nd / nb if nb > 0 else nd, md / mb if mb > 0 else md)
    return float(worst)
