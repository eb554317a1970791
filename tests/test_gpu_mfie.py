"""MFIE part nxK of the electromagnetic listing and its combined system
-beta T + (1 - beta)(Id/2 - nxK) on the GPU (gyps_mfie_apply, gyps_emcfie_apply,
gyps_rhs_planewave_emcfie, GMRES formulation 4) against the oracle, and the
combined-field current's far field against the Mie series."""
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
}


@pytest.fixture(scope="module", params=list(MESHES))
def pair(request, g):
    v, t, q = MESHES[request.param]()
    return g.Mesh(v, t, q), oracle.EfieMesh(v, t, q)


@pytest.mark.parametrize("k", [2.0, 6.0])
@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_mfie_apply_vs_oracle(g, pair, k, nrhs, prec, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(nrhs + 41), om.ne, nrhs)
    y = g.mfie_apply(gm, k, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.mfie_apply(k, x)) < tol


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_emcfie_apply_vs_oracle(g, pair, beta, prec, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(9), om.ne, 2)
    y = g.emcfie_apply(gm, 3.0, beta, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.emcfie_apply(3.0, beta, x)) < tol


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_rhs_planewave_emcfie_vs_oracle(g, pair, beta):
    gm, om = pair
    dirs = synth.plane_wave_dirs(np.random.default_rng(5), 2)
    pols = np.cross(dirs, synth.plane_wave_dirs(np.random.default_rng(6), 2))
    f = g.rhs_planewave_emcfie(gm, 4.0, beta, dirs, pols).cpu().numpy()
    assert rel(f, om.rhs_planewave_emcfie(4.0, beta, dirs, pols)) < 1e-12


def test_mfie_host_buffers_and_errors(g, pair):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(3), om.ne, 2)
    yh = g.emcfie_apply(gm, 3.0, 0.3, torch.as_tensor(x), prec="fp64")
    yd = g.emcfie_apply(gm, 3.0, 0.3, torch.as_tensor(x).cuda(), prec="fp64").cpu()
    assert not yh.is_cuda and rel(yh.numpy(), yd.numpy()) < 1e-13
    for fn, args, status in ((g.mfie_apply, (0.0,), "INVALID"), (g.emcfie_apply, (3.0, float("nan")), "INVALID")):
        with pytest.raises(g.GypsError) as e:
            fn(gm, *args, torch.as_tensor(x).cuda())
        assert e.value.status == status
    with pytest.raises(g.GypsError) as e:
        g.mfie_apply(gm, 3.0, torch.as_tensor(x).cuda(), prec="tc_bf16x3")
    assert e.value.status == "UNSUPPORTED"


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_emcfie_gmres_pec_sphere(g, prec):
    """The listing's system at beta = 0.5 on the unit sphere (k = 2, x-polarised wave
    along z): GMRES matches the oracle's solve, the far field is within 4 % of the Mie
    amplitudes, and it takes fewer iterations than the EFIE."""
    v, t = synth.icosphere(3)
    gm, om = g.Mesh(v, t, 3), oracle.EfieMesh(v, t, 3)
    k, d, p = 2.0, np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    F = g.rhs_planewave_emcfie(gm, k, 0.5, d[None, :], p[None, :])
    x, rep = g.gmres_solve(gm, k, F, tol=1e-8, restart=300, maxit=1000, prec=prec, check_prec="fp64",
                           formulation="emcfie", eta=0.5)
    assert rep.status == "OK" and rep.converged.all()
    xn = x.cpu().numpy()[:, 0]
    f = om.rhs_planewave_emcfie(k, 0.5, d, p)[:, 0]
    assert np.linalg.norm(om.emcfie_apply(k, 0.5, xn) - f) / np.linalg.norm(f) < 2e-8
    xo, _, _ = oracle.gmres(lambda z: om.emcfie_apply(k, 0.5, z), f, tol=1e-10, restart=300, maxit=3000)
    assert np.linalg.norm(xn - xo) / np.linalg.norm(xo) < 1e-6
    th = np.linspace(0.05, np.pi - 0.05, 12)
    s1, s2 = oracle.mie_pec_amplitudes(k, np.cos(th))
    J = np.stack([om.rwg[c] @ xn for c in range(3)], axis=1)
    for xd, s in ((np.stack([np.sin(th), 0 * th, np.cos(th)], 1), s2), (np.stack([0 * th, np.sin(th), np.cos(th)], 1), s1)):
        I = np.exp(-1j * k * (xd @ om.x.T)) @ (om.w[:, None] * J)
        amp = k / (4.0 * np.pi) * np.linalg.norm(I - np.sum(I * xd, axis=1)[:, None] * xd, axis=1)
        assert np.abs(amp / (np.abs(s) / k) - 1.0).max() < 0.04
    Fe = g.rhs_planewave_efie(gm, k, d[None, :], p[None, :])
    _, re = g.gmres_solve(gm, k, Fe, tol=1e-8, restart=300, maxit=1000, prec=prec, check_prec="fp64",
                          formulation="efie")
    assert re.converged.all() and re.iterations > rep.iterations
