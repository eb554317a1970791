"""Pins of the oracle's double layer (the next operator after the single
layer: the paper's grady[exp(ikr)/r] kernel with the 'grady[1/r]'
regularisation), K_ij = (1/4pi) int int phi_i(x) n_y . grad_y exp(ik|x-y|)/|x-y| phi_j(y)."""
import numpy as np
import pytest
from scipy.special import eval_legendre, spherical_jn, spherical_yn

import oracle
import synth
from quadrature_ref import inner_integral

TRI = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.3, 0.8, 0.0])]


@pytest.mark.parametrize("x", [[0.4, 0.3, 0.5], [0.4, 0.3, -0.1], [1.5, -0.4, 0.2], [0.2, 0.1, 0.02],
                               [0.5, -0.3, -0.7], [0.5, 0.0, 0.05], [0.0, 0.0, 0.3], [3.0, 2.0, -1.0]])
def test_p1_dn_inv_r_vs_duffy(x):
    """Closed form against polar (Duffy) Gauss-Legendre quadrature of lambda_j h / R^3."""
    x = np.array(x)
    ref = inner_integral(x, TRI, lambda R: x[2] / R ** 3, ng=80)
    assert np.abs(oracle.p1_dn_inv_r(x, *TRI) - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_p1_dn_inv_r_sums_to_the_solid_angle():
    """sum_j lambda_j = 1: the three values add up to the signed solid angle of
    the triangle (Van Oosterom and Strackee 1983), and vanish in its plane."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.normal(size=3) * 0.8 + np.array([0.4, 0.3, 0.0])
        a, b, c = (p - x for p in TRI)
        la, lb, lc = (np.linalg.norm(v) for v in (a, b, c))
        num = np.dot(a, np.cross(b, c))
        den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
        omega = -2.0 * np.arctan2(num, den)  # num = -h x (2 area) for the normal (P1 - P0) x (P2 - P0)
        assert abs(oracle.p1_dn_inv_r(x, *TRI).sum() - omega) < 1e-12
    assert np.abs(oracle.p1_dn_inv_r(np.array([0.4, 0.3, 0.0]), *TRI)).max() == 0.0


def _mu(n, k):
    """Double-layer eigenvalue on the unit sphere for degree-n harmonics (outward
    normal): -1/(2(2n+1)) at k = 0, else 1/2 + i k^2 j_n(k) h_n'(k)."""
    if k == 0.0:
        return -1.0 / (2 * (2 * n + 1))
    hp = spherical_jn(n, k, derivative=True) + 1j * spherical_yn(n, k, derivative=True)
    return 0.5 + 1j * k * k * spherical_jn(n, k) * hp


@pytest.mark.parametrize("k", [0.0, 5.0])
@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_double_layer_sphere_eigenvalues(k, n):
    """K u = mu_n M u for P1 interpolants of zonal harmonics; the error shrinks
    under refinement (O(h^2) at k = 5, below 2e-3 at every level for k = 0,
    where the constant density gives Gauss's law K 1 = -M 1 / 2)."""
    errs = []
    for level in (2, 3, 4):
        v, t = synth.icosphere(level)
        m = oracle.Mesh(v, t, 3)
        u = eval_legendre(n, v[:, 2] / np.linalg.norm(v, axis=1)).astype(complex)
        mu_ = m.mass() @ u
        errs.append(np.linalg.norm(m.dl_apply(k, u) - _mu(n, k) * mu_) / np.linalg.norm(mu_))
    assert errs[2] < errs[1] < errs[0], errs
    if k > 0.0:
        assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0 and errs[2] < 5e-3, errs
    else:
        assert errs[0] < 2e-3, errs


@pytest.mark.parametrize("shared", ["edge", "vertex"])
def test_adjacent_pair_double_layer_vs_brute_force(shared):
    """Two triangles sharing an edge (or a vertex), out of plane: the whole K
    (far part + correction) against the same outer rule with Duffy inner
    integrals of (1 - ikr) exp(ikr) h / r^3; O(h^2)."""
    k = 4.0
    errs = []
    for h in (0.1, 0.05):
        P = np.array([[0.0, 0.0, 0.0], [h, 0.0, 0.0], [0.4 * h, 0.9 * h, 0.0], [0.6 * h, -0.8 * h, 0.3 * h],
                      [-0.7 * h, -0.2 * h, 0.25 * h], [-0.3 * h, -0.9 * h, -0.15 * h]])
        tri = np.array([[0, 1, 2], [1, 0, 3]] if shared == "edge" else [[0, 1, 2], [0, 4, 5]], dtype=np.int32)
        used = np.unique(tri)
        tri = np.searchsorted(used, tri).astype(np.int32)
        P = P[used]
        m = oracle.Mesh(P, tri, 7)
        K = np.stack([m.dl_apply(k, e) for e in np.eye(m.nv, dtype=complex)], axis=1)
        bary, _ = oracle.quad_rule(7)
        ref = np.zeros_like(K)
        for a in range(2):
            for b in range(2):
                if a == b:
                    continue  # coplanar: the kernel vanishes
                Pb = [P[v] for v in tri[b]]
                nb = np.cross(Pb[1] - Pb[0], Pb[2] - Pb[0])
                nb /= np.linalg.norm(nb)
                for kk in range(7):
                    xk = m.x[7 * a + kk]
                    hh = np.dot(nb, xk - Pb[0])
                    inner = inner_integral(xk, Pb, lambda r: (1 - 1j * k * r) * np.exp(1j * k * r) * hh / r ** 3, ng=80)
                    ref[np.ix_(tri[a], tri[b])] += m.w[7 * a + kk] * np.outer(bary[kk], inner) / (4 * np.pi)
        errs.append(np.abs(K - ref).max() / np.abs(ref).max())
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 3.5, errs
