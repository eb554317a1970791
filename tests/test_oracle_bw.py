"""Pins of the oracle's Brakhage-Werner combined operator 1/2 M + K - i eta V
(the indirect combined-field formulation built from the single and double
layers), on the unit sphere at the resonant wavenumber k = pi, where j_0(k) = 0
and the first-kind operator V has a zero eigenvalue."""
import numpy as np
import pytest
from scipy.special import eval_legendre, spherical_jn, spherical_yn

import oracle
import synth

D = np.array([0.0, 0.0, 1.0])


def _solve_bw(m, k, eta):
    f = m.rhs_planewave(k, D[None, :])[:, 0]
    x, _, res = oracle.gmres(lambda z: m.bw_apply(k, eta, z), -f, tol=1e-10, restart=200)
    assert res < 1e-9
    return x


def _mie_far_field(k, c):
    """Far-field pattern of the sound-soft sphere, u_sca ~ exp(ikr)/r F(cos theta):
    F = (i/k) sum_n (2n+1) j_n(k)/h_n(k) P_n(cos theta) (separation of variables)."""
    nmax = int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 10))
    f = np.zeros_like(c, dtype=np.complex128)
    for n in range(nmax + 1):
        h = spherical_jn(n, k) + 1j * spherical_yn(n, k)
        f += (2 * n + 1) * spherical_jn(n, k) / h * eval_legendre(n, c)
    return 1j / k * f


@pytest.fixture(scope="module")
def levels():
    out = {}
    for level in (2, 3):
        v, t = synth.icosphere(level)
        m = oracle.Mesh(v, t, 3)
        out[level] = (v, m, _solve_bw(m, np.pi, np.pi))
    return out


def test_bw_density_matches_the_closed_form(levels):
    """phi_n = -(2n+1) i^n j_n(k) / (1/2 + mu_n(K) - i eta mu_n(V)) per harmonic;
    the P1 solution converges at O(h^2)."""
    errs = []
    for level in (2, 3):
        v, m, x = levels[level]
        ref = oracle.bw_density(np.pi, np.pi, D, v)
        errs.append(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert errs[1] < 0.02 and errs[0] / errs[1] > 3.0, errs


def test_bw_far_field_matches_mie(levels):
    """The represented field u = (D - i eta S) phi has the far field
    (1/4pi) int (-ik xh.n_y - i eta) exp(-ik xh.y) phi(y): it must be the Mie
    pattern of the sound-soft sphere (which fixes the jump term, the sign of the
    double layer and of i eta), converging at O(h^2)."""
    th = np.linspace(0.0, np.pi, 13)
    xh = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], axis=1)
    fm = _mie_far_field(np.pi, xh @ D)
    errs = []
    for level in (2, 3):
        _, m, x = levels[level]
        e = np.exp(-1j * np.pi * (xh @ m.x.T))
        kern = e * (-1j * np.pi * (xh @ m.point_normals().T) - 1j * np.pi)
        f = kern @ (m.w * (m.phi @ x)) / (4.0 * np.pi)
        errs.append(np.abs(f - fm).max() / np.abs(fm).max())
    assert errs[1] < 6e-3 and errs[0] / errs[1] > 3.0, errs


def test_bw_reduces_to_its_parts():
    """eta = 0 leaves 1/2 M + K; a zero density maps to zero; the operator is linear in eta."""
    v, t = synth.icosphere(1)
    m = oracle.Mesh(v, t, 3)
    x = synth.random_complex(np.random.default_rng(2), m.nv, 2)
    a0 = m.bw_apply(2.0, 0.0, x)
    assert np.abs(a0 - (0.5 * (m.mass() @ x) + m.dl_apply(2.0, x))).max() < 1e-13 * np.abs(a0).max()
    a1 = m.bw_apply(2.0, 1.0, x)
    a3 = m.bw_apply(2.0, 3.0, x)
    assert np.abs((a3 - a0) - 3.0 * (a1 - a0)).max() < 1e-12 * np.abs(a3).max()
    assert np.abs(m.bw_apply(2.0, 1.0, np.zeros((m.nv, 1)))).max() == 0.0
