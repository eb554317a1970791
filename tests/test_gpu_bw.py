"""Brakhage-Werner combined operator (gyps_bw_apply) and the combined-field
GMRES solve against the oracle: operator parity per precision, the sphere
density at the resonant wavenumber k = pi, and the first-kind solve beside it."""
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


@pytest.fixture(scope="module")
def ell(g):
    v, t = synth.ellipsoid(2, (0.7, 1.1, 1.4), (0.3, -0.2, 1.0), 0.6)
    return g.Mesh(v, t, 3), oracle.Mesh(v, t, 3)


@pytest.fixture(scope="module")
def sph(g):
    v, t = synth.icosphere(3)
    return v, g.Mesh(v, t, 3), oracle.Mesh(v, t, 3)


@pytest.mark.parametrize("k,eta", [(0.0, 1.0), (6.0, 6.0), (6.0, 0.0)])
@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_bw_apply_vs_oracle(g, ell, k, eta, nrhs, prec, tol):
    gm, om = ell
    x = synth.random_complex(np.random.default_rng(nrhs + 11), om.nv, nrhs)
    y = g.bw_apply(gm, k, eta, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.bw_apply(k, eta, x)) < tol


def test_bw_apply_tensor_cores(g, ell):
    gm, om = ell
    x = synth.random_complex(np.random.default_rng(5), om.nv, 16)
    y = g.bw_apply(gm, 6.0, 6.0, torch.as_tensor(x).cuda(), prec="tc_bf16x3").cpu().numpy()
    assert rel(y, om.bw_apply(6.0, 6.0, x)) < 1e-5


def test_bw_apply_host_buffers_and_errors(g, ell):
    gm, om = ell
    x = synth.random_complex(np.random.default_rng(0), om.nv, 2)
    yh = g.bw_apply(gm, 3.0, 2.0, torch.as_tensor(x), prec="fp64")
    yd = g.bw_apply(gm, 3.0, 2.0, torch.as_tensor(x).cuda(), prec="fp64").cpu()
    assert not yh.is_cuda and rel(yh.numpy(), yd.numpy()) < 1e-13
    with pytest.raises(g.GypsError) as e:
        g.bw_apply(gm, 3.0, float("nan"), torch.as_tensor(x).cuda())
    assert e.value.status == "INVALID"
    with pytest.raises(g.GypsError) as e:
        g.bw_apply(gm, 3.0, 1.0, torch.as_tensor(x).cuda(), prec="tc_bf16x3")
    assert e.value.status == "UNSUPPORTED"


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bw_gmres_sphere_at_resonance(g, sph, prec):
    """k = pi on the unit sphere: the combined-field solve reaches 1e-8 against
    the oracle operator and matches the oracle's own solution and the closed
    form; the first-kind solve of the same problem needs more iterations."""
    v, gm, om = sph
    k = np.pi
    F = g.rhs_planewave(gm, k, D[None, :])
    x, rep = g.gmres_solve(gm, k, -F, tol=1e-8, restart=200, maxit=400, prec=prec, check_prec="fp64",
                           formulation="bw", eta=k)
    assert rep.status == "OK" and rep.converged.all()
    xn = x.cpu().numpy()
    f = om.rhs_planewave(k, D[None, :])
    r = om.bw_apply(k, k, xn) + f
    assert np.linalg.norm(r) / np.linalg.norm(f) < 2e-8
    xo, _, _ = oracle.gmres(lambda z: om.bw_apply(k, k, z), -f[:, 0], tol=1e-10, restart=200)
    assert np.linalg.norm(xn[:, 0] - xo) / np.linalg.norm(xo) < 1e-6
    ref = oracle.bw_density(k, k, D, v)
    assert np.linalg.norm(xn[:, 0] - ref) / np.linalg.norm(ref) < 0.02
    _, rsl = g.gmres_solve(gm, k, F, tol=1e-8, restart=200, maxit=400, prec=prec, check_prec="fp64")
    assert rsl.converged.all() and rsl.iterations > rep.iterations


def test_bw_gmres_host_input_and_several_columns(g, ell):
    gm, om = ell
    k = 5.0
    dirs = synth.plane_wave_dirs(np.random.default_rng(3), 3)
    F = om.rhs_planewave(k, dirs)
    x, rep = g.gmres_solve(gm, k, torch.as_tensor(-F), tol=1e-8, restart=100, maxit=300, prec="fp32",
                           formulation="bw", eta=2.0)
    assert rep.converged.all() and not x.is_cuda
    r = om.bw_apply(k, 2.0, x.numpy()) + F
    for c in range(3):
        assert np.linalg.norm(r[:, c]) / np.linalg.norm(F[:, c]) < 2e-8


def test_bw_gmres_option_errors(g, ell):
    gm, om = ell
    F = torch.as_tensor(om.rhs_planewave(2.0, np.eye(3)[:1])).cuda()
    with pytest.raises(g.GypsError) as e:
        g.gmres_solve(gm, 2.0, F, formulation="bw", eta=float("inf"), raise_on_fail=True)
    assert e.value.status == "INVALID"
    p = g.Precond(64, 2, 1)
    with pytest.raises(g.GypsError) as e:
        g.gmres_solve(gm, 2.0, F, formulation="bw", precond=p, raise_on_fail=True)
    assert e.value.status == "UNSUPPORTED"
