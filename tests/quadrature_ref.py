"""Independent numerical integration used to pin the oracle (tests only).

Inner integrals over a flat triangle are evaluated by splitting the triangle
into three sub-triangles with apex at the in-plane projection of the
observation point and mapping each with the Duffy transform, so that the 1/r
singularity is cancelled by the Jacobian; a tensor Gauss-Legendre rule of
order ``ng`` is then applied.  Sub-triangles carry signed areas, so the apex
may lie outside the triangle.
"""
import numpy as np
from numpy.polynomial.legendre import leggauss


def barycentric(P, Y):
    """Barycentric coordinates of points Y (n, 3) in the triangle P (3 x 3)."""
    m = np.vstack([np.asarray(P, dtype=np.float64).T, np.ones(3)])
    rhs = np.concatenate([Y.T, np.ones((1, Y.shape[0]))])
    return np.linalg.pinv(m) @ rhs  # (3, n)


def inner_integral(x, P, f, ng=60):
    """int_T lambda_j(y) f(|x - y|) dy for j = 0, 1, 2 (f vectorised)."""
    P = [np.asarray(p, dtype=np.float64) for p in P]
    x = np.asarray(x, dtype=np.float64)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    d = (x - P[0]) @ n
    rho = x - d * n
    g, wg = leggauss(ng)
    g = (g + 1) / 2
    wg = wg / 2
    U, V = np.meshgrid(g, g, indexing="ij")
    W = np.outer(wg, wg)
    tot = np.zeros(3, dtype=np.result_type(f(np.array([1.0])), np.float64))
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        s = 0.5 * (np.cross(a - rho, b - rho) @ n)
        Y = rho[None, None, :] + U[..., None] * (a - rho) + (U * V)[..., None] * (b - a)
        R = np.linalg.norm(Y - x, axis=-1)
        jac = 2.0 * s * U
        lam = barycentric(P, Y.reshape(-1, 3))
        tot = tot + lam @ (W * jac * f(R)).reshape(-1)
    return tot


def monomial_integral(area, a, b, c):
    """int_T l1^a l2^b l3^c = 2 area a! b! c! / (a + b + c + 2)!."""
    from math import factorial
    return 2.0 * area * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)


def inner_integral_vec(x, P, ng=60):
    """int_T lambda_j(y) (x - y)/|x - y|^3 dy for j = 0, 1, 2: (3, 3), row j (the same
    Duffy split about the projection of x)."""
    P = [np.asarray(p, dtype=np.float64) for p in P]
    x = np.asarray(x, dtype=np.float64)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    d = (x - P[0]) @ n
    rho = x - d * n
    g, wg = leggauss(ng)
    g = (g + 1) / 2
    wg = wg / 2
    U, V = np.meshgrid(g, g, indexing="ij")
    W = np.outer(wg, wg)
    tot = np.zeros((3, 3))
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        s = 0.5 * (np.cross(a - rho, b - rho) @ n)
        Y = rho[None, None, :] + U[..., None] * (a - rho) + (U * V)[..., None] * (b - a)
        D = x - Y
        R = np.linalg.norm(D, axis=-1)
        jac = 2.0 * s * U
        lam = barycentric(P, Y.reshape(-1, 3))                  # (3, n)
        f = (W * jac / R ** 3)[..., None] * D                  # (ng, ng, 3)
        tot = tot + lam @ f.reshape(-1, 3)
    return tot
