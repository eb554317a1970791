"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds only input generation: meshes, plane-wave directions and
wavenumbers.  It holds none of the single-layer operator's arithmetic
(quadrature, kernel, correction, solve).  The paper's sound-soft sphere test
case (Sec. 5.4) meshes the unit sphere with ``mshSphere``, whose construction
is not given; an icosphere stands in for it, and random-axis ellipsoids made by
mapping icosphere vertices stand in for the uneven batch of meshes.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "icosphere",
    "ellipsoid",
    "random_ellipsoid",
    "plane_wave_dirs",
    "unit_sphere_counts",
    "random_complex",
    "WORKLOADS",
]


def _icosahedron():
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
            [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
            [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def _orient_outward(v, f):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, a + b + c) < 0
    f = f.copy()
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return f


def icosphere(level: int, radius: float = 1.0):
    """Icosahedron refined ``level`` times by edge midpoints, projected to the sphere.

    Returns ``(vtx, tri)``: ``vtx`` float64 (Nv, 3), ``tri`` int32 (Nt, 3),
    outward oriented, with Nt = 20*4**level and Nv = 10*4**level + 2.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = _icosahedron()
    f = _orient_outward(v, f)
    for _ in range(level):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        uk, inv = np.unique(key, return_inverse=True)
        ea, eb = uk // (nv + 1), uk % (nv + 1)
        mid = 0.5 * (v[ea] + v[eb])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate(
            [
                np.stack([a, m01, m20], 1),
                np.stack([b, m12, m01], 1),
                np.stack([c, m20, m12], 1),
                np.stack([m01, m12, m20], 1),
            ],
            axis=0,
        )
    return np.ascontiguousarray(v * radius), np.ascontiguousarray(f.astype(np.int32))


def unit_sphere_counts(level: int):
    """(Nv, Nt) of an icosphere of the given level."""
    return 10 * 4 ** level + 2, 20 * 4 ** level


def _rotation(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    kx = np.array([[0, -z, y], [z, 0, -x], [-y, x, 0]])
    return np.eye(3) + np.sin(angle) * kx + (1 - np.cos(angle)) * kx @ kx


def ellipsoid(level: int, semi_axes, axis=(0.0, 0.0, 1.0), angle: float = 0.0):
    """Icosphere vertices mapped by v -> R diag(a, b, c) v (R: rotation about ``axis``)."""
    v, f = icosphere(level)
    rot = _rotation(axis, angle)
    v = (v * np.asarray(semi_axes, dtype=np.float64)[None, :]) @ rot.T
    return np.ascontiguousarray(v), f


def random_ellipsoid(rng: np.random.Generator, level: int, lo: float = 0.5, hi: float = 2.0):
    """Random-axis ellipsoid with semi-axes drawn from U[lo, hi]."""
    ax = rng.uniform(lo, hi, size=3)
    axis = rng.normal(size=3)
    angle = rng.uniform(0.0, 2.0 * np.pi)
    v, f = ellipsoid(level, ax, axis, angle)
    return v, f, ax


def plane_wave_dirs(rng: np.random.Generator, n: int):
    """``n`` directions uniform on the unit sphere (normalised Gaussian draws), shape (n, 3)."""
    d = rng.normal(size=(n, 3))
    return np.ascontiguousarray(d / np.linalg.norm(d, axis=1, keepdims=True))


def random_complex(rng: np.random.Generator, n: int, nrhs: int = 1):
    """Complex (n, nrhs) array with real and imaginary parts from N(0, 1), Fortran order."""
    z = rng.normal(size=(n, nrhs)) + 1j * rng.normal(size=(n, nrhs))
    return np.asfortranarray(z)


# The five workloads of the operator: mesh, quadrature points per triangle,
# wavenumber and right-hand sides.  Sizes follow the sound-soft sphere example
# and the scaling study of the paper (Sec. 6.2, Table 4) on icospheres.
WORKLOADS = {
    "sphere642_k5_q3_dense": dict(level=3, q=3, k=5.0, dirs=[(0.0, 0.0, 1.0)], tol=1e-8),
    "sphere10242_k16_q7": dict(level=5, q=7, k=16.0, dirs=[(1.0, 0.0, 0.0)], tol=1e-6),
    "sphere163842_k64_q3_r16": dict(level=7, q=3, k=64.0, ndirs=16, seed=7, tol=1e-6),
    # EFIE (electromagnetic listing of Sec. 5.5): RWG on the 20480-triangle sphere,
    # x-polarised plane wave along z
    "efie_sphere10242_k8_q3": dict(level=5, q=3, k=8.0, dirs=[(0.0, 0.0, 1.0)], pols=[(1.0, 0.0, 0.0)], tol=1e-6),
}


def j_zeros_near(k: float, delta: float, nmax: int = 80) -> bool:
    """True when k lies within delta of a zero of a spherical Bessel function
    j_n (n <= nmax): the unit sphere's single layer is singular there."""
    from scipy.special import spherical_jn
    xs = np.linspace(max(k - delta, 1e-6), k + delta, 41)
    for n in range(nmax + 1):
        v = spherical_jn(n, xs)
        if np.any(np.sign(v[:-1]) != np.sign(v[1:])):
            return True
    return False


def batch_workload(seed: int = 1804, nrhs: int = 64, levels=(2, 3, 4, 5, 6), n_ellipsoids: int = 7,
                   ell_levels=(2, 6), k_range=(2.0, 24.0)):
    """The uneven batch: icospheres of the given levels plus random-axis
    ellipsoids (level U{ell_levels}, semi-axes U[0.5, 2]); k_i ~ U[k_range],
    redrawn for spheres within 0.02 of a zero of some j_n; nrhs plane-wave
    directions uniform on the sphere.  Returns a list of dicts and the directions."""
    rng = np.random.default_rng(seed)
    items = []
    for lv in levels:
        v, t = icosphere(lv)
        k = rng.uniform(*k_range)
        while j_zeros_near(k, 0.02):
            k = rng.uniform(*k_range)
        items.append(dict(kind="sphere", level=lv, vtx=v, tri=t, k=k))
    for _ in range(n_ellipsoids):
        lv = int(rng.integers(ell_levels[0], ell_levels[1] + 1))
        v, t, ax = random_ellipsoid(rng, lv)
        items.append(dict(kind="ellipsoid", level=lv, vtx=v, tri=t, k=rng.uniform(*k_range), axes=ax))
    dirs = plane_wave_dirs(rng, nrhs)
    return items, dirs
