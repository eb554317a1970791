"""EFIE with RWG functions on the GPU (gyps_rwg_edges, gyps_efie_apply,
gyps_rhs_planewave_efie, GMRES formulation 3) against the oracle, and the solved
current's far field against the Mie series of the perfectly conducting sphere."""
import numpy as np
import pytest

import oracle
import synth
from parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1804_00995_gb300 as g
    return g


MESHES = {
    "ellipsoid_l2_q3": lambda: (*synth.ellipsoid(2, (0.7, 1.1, 1.4), (0.3, -0.2, 1.0), 0.6), 3),
    "sphere_l3_q7": lambda: (*synth.icosphere(3), 7),
    "sphere_l2_q1": lambda: (*synth.icosphere(2), 1),
}


@pytest.fixture(scope="module", params=list(MESHES))
def pair(request, g):
    v, t, q = MESHES[request.param]()
    return g.Mesh(v, t, q), oracle.EfieMesh(v, t, q)


def test_rwg_edges_match_the_oracle(g, pair):
    gm, om = pair
    ne, edges = g.rwg_edges(gm)
    assert ne == om.ne and np.array_equal(edges, om.edges.astype(np.int32))


@pytest.mark.parametrize("k", [2.0, 6.0])
@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_efie_apply_vs_oracle(g, pair, k, nrhs, prec, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(nrhs + 31), om.ne, nrhs)
    y = g.efie_apply(gm, k, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.efie_apply(k, x)) < tol


def test_efie_host_buffers_rhs_and_errors(g, pair):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(2), om.ne, 2)
    yh = g.efie_apply(gm, 3.0, torch.as_tensor(x), prec="fp64")
    yd = g.efie_apply(gm, 3.0, torch.as_tensor(x).cuda(), prec="fp64").cpu()
    assert not yh.is_cuda and rel(yh.numpy(), yd.numpy()) < 1e-13
    dirs = synth.plane_wave_dirs(np.random.default_rng(5), 3)
    pols = np.cross(dirs, synth.plane_wave_dirs(np.random.default_rng(6), 3))
    f = g.rhs_planewave_efie(gm, 4.0, dirs, pols).cpu().numpy()
    assert rel(f, om.rhs_planewave_efie(4.0, dirs, pols)) < 1e-12
    fh = g.rhs_planewave_efie(gm, 4.0, dirs, pols, device="cpu").numpy()
    assert rel(fh, f) < 1e-15
    for kk, prec, status in ((0.0, "fp32", "INVALID"), (3.0, "tc_bf16x3", "UNSUPPORTED")):
        with pytest.raises(g.GypsError) as e:
            g.efie_apply(gm, kk, torch.as_tensor(x).cuda(), prec=prec)
        assert e.value.status == status


def test_rwg_needs_a_closed_mesh(g):
    v, t = synth.icosphere(1)
    gm = g.Mesh(v, t[1:], 3)
    with pytest.raises(g.GypsError) as e:
        g.rwg_edges(gm)
    assert e.value.status == "INVALID"


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_efie_gmres_pec_sphere(g, prec):
    """-T J = int phi . E_inc on the unit sphere (k = 2, x-polarised wave along z):
    the GMRES current matches the oracle's solve and its far field the Mie
    amplitudes of the perfectly conducting sphere."""
    v, t = synth.icosphere(3)
    gm, om = g.Mesh(v, t, 3), oracle.EfieMesh(v, t, 3)
    k, d, p = 2.0, np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    F = g.rhs_planewave_efie(gm, k, d[None, :], p[None, :])
    x, rep = g.gmres_solve(gm, k, F, tol=1e-8, restart=300, maxit=1000, prec=prec, check_prec="fp64",
                           formulation="efie")
    assert rep.status == "OK" and rep.converged.all()
    xn = x.cpu().numpy()[:, 0]
    f = om.rhs_planewave_efie(k, d, p)[:, 0]
    assert np.linalg.norm(-om.efie_apply(k, xn) - f) / np.linalg.norm(f) < 2e-8
    xo, _, _ = oracle.gmres(lambda z: -om.efie_apply(k, z), f, tol=1e-10, restart=300, maxit=3000)
    assert np.linalg.norm(xn - xo) / np.linalg.norm(xo) < 1e-6
    th = np.linspace(0.05, np.pi - 0.05, 12)
    s1, s2 = oracle.mie_pec_amplitudes(k, np.cos(th))
    J = np.stack([om.rwg[c] @ xn for c in range(3)], axis=1)
    for xd, s in ((np.stack([np.sin(th), 0 * th, np.cos(th)], 1), s2), (np.stack([0 * th, np.sin(th), np.cos(th)], 1), s1)):
        I = np.exp(-1j * k * (xd @ om.x.T)) @ (om.w[:, None] * J)
        amp = k / (4.0 * np.pi) * np.linalg.norm(I - np.sum(I * xd, axis=1)[:, None] * xd, axis=1)
        assert np.abs(amp / (np.abs(s) / k) - 1.0).max() < 0.02
