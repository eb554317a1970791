"""Adjoint double layer (gyps_adl_apply), the direct combined-field operator
(gyps_cfie_apply), its right-hand side and the combined-field GMRES solve,
against the oracle; the solve's density against the Mie series at the resonant
k = pi on the unit sphere."""
import numpy as np
import pytest

import oracle
import synth
from parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

D = np.array([0.0, 0.0, 1.0])


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
    return g.Mesh(v, t, q), oracle.Mesh(v, t, q)


@pytest.mark.parametrize("k", [0.0, 6.0])
@pytest.mark.parametrize("nrhs", [1, 3, 9])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_adl_apply_vs_oracle(g, pair, k, nrhs, prec, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(nrhs + 21), om.nv, nrhs)
    y = g.adl_apply(gm, k, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.adl_apply(k, x)) < tol


def test_adl_is_the_transpose_of_dl_on_the_gpu(g):
    v, t = synth.ellipsoid(1, (0.8, 1.0, 1.3), (1.0, 0.0, 0.0), 0.4)
    gm = g.Mesh(v, t, 3)
    eye = torch.eye(gm.nv, dtype=torch.complex128).cuda()
    a = g.dl_apply(gm, 4.0, eye, prec="fp64").cpu().numpy()
    b = g.adl_apply(gm, 4.0, eye, prec="fp64").cpu().numpy()
    assert np.abs(b - a.T).max() < 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("k,eta", [(0.0, 1.0), (6.0, 6.0)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_cfie_apply_vs_oracle(g, pair, k, eta, prec, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(7), om.nv, 2)
    y = g.cfie_apply(gm, k, eta, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.cfie_apply(k, eta, x)) < tol


def test_cfie_apply_tensor_cores(g, pair):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(8), om.nv, 16)
    y = g.cfie_apply(gm, 6.0, 6.0, torch.as_tensor(x).cuda(), prec="tc_bf16x3").cpu().numpy()
    assert rel(y, om.cfie_apply(6.0, 6.0, x)) < 1e-4  # the tensor-core V's bound (split bf16 products)


@pytest.mark.parametrize("k,eta", [(0.0, 1.0), (5.0, 0.0), (5.0, 5.0)])
def test_rhs_planewave_cfie_vs_oracle(g, pair, k, eta):
    gm, om = pair
    dirs = synth.plane_wave_dirs(np.random.default_rng(4), 3)
    f = g.rhs_planewave_cfie(gm, k, eta, dirs).cpu().numpy()
    assert rel(f, om.rhs_planewave_cfie(k, eta, dirs)) < 1e-12
    fh = g.rhs_planewave_cfie(gm, k, eta, dirs, device="cpu").numpy()
    assert rel(fh, f) < 1e-15


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cfie_gmres_sphere_at_resonance(g, prec):
    """k = pi, unit sphere: the combined-field solve reaches 1e-8 against the oracle
    operator, matches the oracle's solve, gives the Mie density d(u)/dn to the
    discretisation error, and needs fewer iterations than the first-kind solve."""
    v, t = synth.icosphere(3)
    gm, om = g.Mesh(v, t, 3), oracle.Mesh(v, t, 3)
    k = np.pi
    F = g.rhs_planewave_cfie(gm, k, k, D[None, :])
    x, rep = g.gmres_solve(gm, k, F, tol=1e-8, restart=200, maxit=400, prec=prec, check_prec="fp64",
                           formulation="cfie", eta=k)
    assert rep.status == "OK" and rep.converged.all()
    xn = x.cpu().numpy()
    f = om.rhs_planewave_cfie(k, k, D[None, :])
    assert np.linalg.norm(om.cfie_apply(k, k, xn) - f) / np.linalg.norm(f) < 2e-8
    xo, _, _ = oracle.gmres(lambda z: om.cfie_apply(k, k, z), f[:, 0], tol=1e-10, restart=200)
    assert np.linalg.norm(xn[:, 0] - xo) / np.linalg.norm(xo) < 1e-6
    ref = oracle.mie_density(k, D, v)
    assert np.linalg.norm(xn[:, 0] - ref) / np.linalg.norm(ref) < 0.02
    Fs = g.rhs_planewave(gm, k, D[None, :])
    _, rsl = g.gmres_solve(gm, k, Fs, tol=1e-8, restart=200, maxit=400, prec=prec, check_prec="fp64")
    assert rsl.converged.all() and rsl.iterations > rep.iterations


def test_cfie_gmres_errors(g, pair):
    gm, om = pair
    F = torch.as_tensor(om.rhs_planewave_cfie(2.0, 2.0, np.eye(3)[:1])).cuda()
    p = g.Precond(64, 2, 1)
    with pytest.raises(g.GypsError) as e:
        g.gmres_solve(gm, 2.0, F, formulation="cfie", precond=p, raise_on_fail=True)
    assert e.value.status == "UNSUPPORTED"
    with pytest.raises(g.GypsError) as e:
        g.rhs_planewave_cfie(gm, 2.0, float("nan"), np.eye(3)[:1])
    assert e.value.status == "INVALID"
