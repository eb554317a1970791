"""Pins of the oracle's MFIE part nxK of the electromagnetic listing of
Sec. 5.5 (kernel grad_y exp(ikr)/r tested with n x phi, 'grady[1/r]'
regularisation) and of the listing's combined system
-beta T + (1 - beta)(Id/2 - nxK)."""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
import synth
from quadrature_ref import inner_integral_vec

TRI = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.3, 0.8, 0.0])]


def _vertex_apex_vec(x, P, ng=200):
    """int_T lambda_j (x - y)/|x - y|^3 by a product Gauss rule with the Duffy apex at
    vertex P0 (for x away from T, where the integrand is smooth)."""
    g, w = leggauss(ng)
    g, w = (g + 1) / 2, w / 2
    U, V = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w)
    A, B, C = P
    Y = A + U[..., None] * (B - A) + (U * V)[..., None] * (C - B)
    jac = np.linalg.norm(np.cross(B - A, C - A)) * U
    D = x - Y
    R = np.linalg.norm(D, axis=-1)
    lam = (1 - U, U * (1 - V), U * V)
    return np.array([((W * jac * l / R ** 3)[..., None] * D).reshape(-1, 3).sum(0) for l in lam])


@pytest.mark.parametrize("x", [[0.4, 0.3, 0.5], [0.4, 0.3, -0.1], [1.5, -0.4, 0.2], [0.2, 0.1, 0.02],
                               [0.5, -0.3, -0.7], [0.5, 0.0, 0.05], [3.0, 2.0, -1.0], [0.4, 0.3, 0.003]])
def test_p1_grad_inv_r_vs_duffy(x):
    x = np.array(x)
    ref = inner_integral_vec(x, TRI, ng=120)
    assert np.abs(oracle.p1_grad_inv_r(x, *TRI) - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("x", [[1.4, 1.2, 0.0], [2.0, -0.5, 0.0], [-0.3, 0.4, 0.0]])
def test_p1_grad_inv_r_in_plane_outside(x):
    """In the plane, outside the triangle: the normal part vanishes and the in-plane
    part matches a quadrature with the apex at a vertex."""
    x = np.array(x)
    out = oracle.p1_grad_inv_r(x, *TRI)
    assert np.abs(out[:, 2]).max() == 0.0
    ref = _vertex_apex_vec(x, TRI)
    assert np.abs(out - ref).max() < 1e-11 * np.abs(ref).max()


def test_mfie_near_blocks_vs_quadrature():
    """For pairs of neighbouring triangles, the Gauss-Gauss far part plus the
    correction equals the Galerkin entry with the same outer rule and the inner
    integral by quadrature alone (Duffy for the singular part, a dense product rule
    for the smooth remainder) to 1e-3; without the correction the error is above 4 %."""
    k = 2.0
    v, t = synth.icosphere(3)
    m = oracle.EfieMesh(v, t, 3)
    q = m.q
    pa, pb = oracle.near_pairs(m.tri, m.nv)
    C = m.mfie_near
    g, w = leggauss(24)
    g, w = (g + 1) / 2, w / 2
    U, V = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w)
    checked = 0
    for a, b in zip(pa, pb):
        if a == b or checked == 6:
            continue
        checked += 1
        A, B = m.vtx[m.tri[a]], m.vtx[m.tri[b]]
        na = np.cross(A[1] - A[0], A[2] - A[0])
        na /= np.linalg.norm(na)
        area2 = np.linalg.norm(np.cross(B[1] - B[0], B[2] - B[0]))
        Y = (B[0] + U[..., None] * (B[1] - B[0]) + (U * V)[..., None] * (B[2] - B[1])).reshape(-1, 3)
        jac = (area2 * U * W).reshape(-1)
        yb, wb = m.x[b * q:(b + 1) * q], m.w[b * q:(b + 1) * q]
        acc = np.zeros((3, 3), dtype=complex)
        dis = np.zeros((3, 3), dtype=complex)
        for kk in range(q):
            x, wk = m.x[a * q + kk], m.w[a * q + kk]
            Vs = inner_integral_vec(x, B, ng=60)                  # int lambda_m (x - y)/R^3
            D = x - Y
            r = np.linalg.norm(D, axis=1)
            fs = ((1 - 1j * k * r) * np.exp(1j * k * r) - 1) / r ** 3
            Dg = x - yb
            rg = np.linalg.norm(Dg, axis=1)
            fg = (1 - 1j * k * rg) * np.exp(1j * k * rg) / rg ** 3
            for j in range(3):
                cj = m.tsign[b, j] * np.linalg.norm(B[(j + 2) % 3] - B[(j + 1) % 3]) / area2
                fj, _ = oracle.rwg_eval(B, j, m.tsign[b, j], Y)
                inner = ((jac * fs)[:, None] * np.cross(D, fj)).sum(0)
                inner = inner + cj * sum(np.cross(Vs[mm], B[mm] - B[j]) for mm in range(3))
                fjg, _ = oracle.rwg_eval(B, j, m.tsign[b, j], yb)
                gauss = ((wb * fg)[:, None] * np.cross(Dg, fjg)).sum(0)
                for i in range(3):
                    fi, _ = oracle.rwg_eval(A, i, m.tsign[a, i], x)
                    tf = np.cross(na, fi[0])
                    acc[i, j] += wk * tf @ inner / (4 * np.pi)
                    dis[i, j] += wk * tf @ gauss / (4 * np.pi)
        # the correction of this pair alone, from the pair's own blocks
        blk = np.zeros((3, 3))
        lib = oracle._load()
        tsg = np.ascontiguousarray(m.tsign)
        one_a, one_b = np.array([a], dtype=np.int64), np.array([b], dtype=np.int64)
        lib.or_mfie_near_blocks(oracle._dp(np.ascontiguousarray(m.vtx)),
                                oracle._i32p(np.ascontiguousarray(m.tri, dtype=np.int32)), oracle._dp(tsg), q, 1,
                                oracle._i64p(one_a), oracle._i64p(one_b), oracle._dp(blk))
        scale = np.abs(acc).max()
        assert np.abs(dis + blk - acc).max() < 1e-3 * scale
        assert np.abs(dis - acc).max() > 4e-2 * scale
    assert checked == 6
    assert C.shape == (m.ne, m.ne)


def _mie_error(m, k, x):
    th = np.linspace(0.05, np.pi - 0.05, 12)
    s1, s2 = oracle.mie_pec_amplitudes(k, np.cos(th))
    J = np.stack([m.rwg[c] @ x for c in range(3)], axis=1)
    err = 0.0
    for xd, s in ((np.stack([np.sin(th), 0 * th, np.cos(th)], 1), s2), (np.stack([0 * th, np.sin(th), np.cos(th)], 1), s1)):
        I = np.exp(-1j * k * (xd @ m.x.T)) @ (m.w[:, None] * J)
        amp = k / (4.0 * np.pi) * np.linalg.norm(I - np.sum(I * xd, axis=1)[:, None] * xd, axis=1)
        err = max(err, np.abs(amp / (np.abs(s) / k) - 1.0).max())
    return err


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_mfie_and_cfie_pec_sphere_far_field(beta):
    """The listing's system at beta = 0 (MFIE) and 0.5 on the unit sphere, k = 2,
    x-polarised wave along z: the far field converges to the Mie amplitudes of the
    perfectly conducting sphere (a flipped nxK gives 53 % at the finer level), and the
    MFIE, a second-kind equation, needs far fewer iterations than the EFIE."""
    k, d, p = 2.0, np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    errs, its = [], []
    for level in (2, 3):
        v, t = synth.icosphere(level)
        m = oracle.EfieMesh(v, t, 3)
        f = m.rhs_planewave_emcfie(k, beta, d, p)[:, 0]
        x, it, res = oracle.gmres(lambda z: m.emcfie_apply(k, beta, z), f, tol=1e-8, restart=300, maxit=3000)
        assert res < 1e-7
        errs.append(_mie_error(m, k, x))
        its.append(it)
    assert errs[1] < 0.04 and errs[0] / errs[1] > 2.5, errs
    if beta == 0.0:
        assert max(its) < 25, its
