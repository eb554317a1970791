"""Pins of the oracle's adjoint double layer K' (normal derivative at the test
point) and of the direct combined-field system (1/2 M + K' - i eta V) lambda =
int phi (d/dn - i eta) u_inc, whose solution is the density of the paper's
sound-soft problem (Sec. 5.4), on the unit sphere at the resonant k = pi."""
import numpy as np
import pytest

import oracle
import synth

D = np.array([0.0, 0.0, 1.0])


def test_adjoint_double_layer_is_the_transpose():
    """G is symmetric, so the Galerkin K' is K^T; the oracle evaluates K' with its
    own kernel (normal at the target), which must give the transpose of K."""
    v, t = synth.icosphere(1)
    m = oracle.Mesh(v, t, 3)
    eye = np.eye(m.nv)
    a = m.dl_apply(3.0, eye)
    b = m.adl_apply(3.0, eye)
    assert np.abs(b - a.T).max() < 1e-13 * np.abs(a).max()
    assert np.abs(b - a).max() > 1e-3 * np.abs(a).max()  # K itself is not symmetric on this mesh


@pytest.mark.parametrize("eta", [0.0, 1.5])
def test_cfie_rhs_against_the_divergence_theorem(eta):
    """sum_i F_i = int_S (d/dn - i eta) exp(ik d.x): by Gauss, int_S d/dn exp(ik d.x) =
    -k^2 int_B exp(ik d.x) = -4 pi (sin k - k cos k)/k, and int_S exp(ik d.x) = 4 pi sin(k)/k
    on the unit sphere; the P1 sums converge at O(h^2)."""
    k = 2.0
    exact = -4.0 * np.pi * (np.sin(k) - k * np.cos(k)) / k - 1j * eta * 4.0 * np.pi * np.sin(k) / k
    errs = []
    for level in (2, 3, 4):
        v, t = synth.icosphere(level)
        m = oracle.Mesh(v, t, 3)
        errs.append(abs(m.rhs_planewave_cfie(k, eta, D[None, :]).sum() - exact) / abs(exact))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5 and errs[2] < 2e-3, errs


def test_cfie_solution_is_the_sound_soft_density():
    """At k = pi the direct combined-field solution converges to the Mie density
    d(u_inc + u_sca)/dn (the same closed form as the first-kind density) at
    O(h^2) and approaches the first-kind Galerkin solution."""
    k = np.pi
    errs, diffs = [], []
    for level in (2, 3):
        v, t = synth.icosphere(level)
        m = oracle.Mesh(v, t, 3)
        f = m.rhs_planewave_cfie(k, k, D[None, :])[:, 0]
        x, _, res = oracle.gmres(lambda z: m.cfie_apply(k, k, z), f, tol=1e-10, restart=200)
        assert res < 1e-9
        ref = oracle.mie_density(k, D, v)
        errs.append(np.linalg.norm(x - ref) / np.linalg.norm(ref))
        fs = m.rhs_planewave(k, D[None, :])[:, 0]
        xs, _, _ = oracle.gmres(lambda z: m.apply(k, z), fs, tol=1e-10, restart=200)
        diffs.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    assert errs[1] < 0.02 and errs[0] / errs[1] > 3.5, errs
    assert diffs[1] < 2e-3 and diffs[0] / diffs[1] > 3.0, diffs
