"""Single-layer potential at points (gyps_sl_potential, the radiation operator
of the listing in Sec. 5.4) against the oracle: FP64 and double-float 1e-10,
FP32 1e-5, with points inside, outside and within 1e-3 of the surface."""
import numpy as np
import pytest

import oracle
import synth
from parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _points(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.concatenate([rng.uniform(0.2, 0.9, n // 3), rng.uniform(1.1, 3.0, n // 3),
                        1.0 + rng.choice([-1e-3, 1e-3, -2e-2, 2e-2], n - 2 * (n // 3))])
    return d * r[:, None]


@pytest.fixture(scope="module")
def g():
    import paper_1804_00995_gb300 as g
    return g


@pytest.fixture(scope="module")
def meshes(g):
    v, t = synth.ellipsoid(2, (0.9, 1.0, 1.1), (0.2, 1.0, 0.3), 0.4)
    return g.Mesh(v, t, 3), oracle.Mesh(v, t, 3), v


@pytest.mark.parametrize("k", [0.0, 5.0])
@pytest.mark.parametrize("nrhs", [1, 5])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_potential_vs_oracle(g, meshes, k, nrhs, prec, tol):
    gm, om, v = meshes
    pts = _points(150, 7 + nrhs)
    x = synth.random_complex(np.random.default_rng(nrhs), om.nv, nrhs)
    got = g.sl_potential(gm, k, torch.as_tensor(pts).cuda(), torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert got.shape == (len(pts), nrhs)
    assert rel(got, om.potential(k, pts, x)) < tol


def test_potential_host_buffers_and_edge_cases(g, meshes):
    gm, om, v = meshes
    pts = _points(40, 3)
    x = synth.random_complex(np.random.default_rng(0), om.nv, 2)
    host = g.sl_potential(gm, 4.0, pts, torch.as_tensor(x), prec="fp64")
    assert not host.is_cuda
    dev = g.sl_potential(gm, 4.0, torch.as_tensor(pts).cuda(), torch.as_tensor(x).cuda(), prec="fp64").cpu()
    assert rel(host.numpy(), dev.numpy()) < 1e-13
    empty = g.sl_potential(gm, 4.0, np.zeros((0, 3)), torch.as_tensor(x).cuda())
    assert empty.shape == (0, 2)
    with pytest.raises(g.GypsError) as e:
        g.sl_potential(gm, 4.0, pts, torch.as_tensor(x).cuda(), prec="tc_bf16x3")
    assert e.value.status == "UNSUPPORTED"
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(g.GypsError) as e:
        g.sl_potential(gm, 4.0, bad, torch.as_tensor(x).cuda())
    assert e.value.status == "INVALID"


def test_total_field_of_the_solved_sphere(g):
    """Sound-soft sphere (icosphere 1280 triangles, k = 5): GMRES density, then
    the total field p_inc - S lambda vanishes inside and matches the Mie field
    outside to the discretisation error, as the oracle's does."""
    v, t = synth.icosphere(3)
    gm = g.Mesh(v, t, 3)
    om = oracle.Mesh(v, t, 3)
    d = (0.0, 0.0, 1.0)
    f = g.rhs_planewave(gm, 5.0, [d])
    lam, rep = g.gmres_solve(gm, 5.0, f, tol=1e-8, restart=200, prec="fp32", check_prec="df64")
    assert rep.status == "OK"
    pts = _points(60, 11)
    pts = pts[np.abs(np.linalg.norm(pts, axis=1) - 1.0) > 0.05]
    p = g.sl_potential(gm, 5.0, torch.as_tensor(pts).cuda(), lam, prec="fp32").cpu().numpy()[:, 0]
    ref = om.potential(5.0, pts, lam.cpu().numpy()[:, 0])
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) < 1e-5
    total = np.exp(1j * 5.0 * pts @ np.array(d)) - p
    inside = np.linalg.norm(pts, axis=1) < 1.0
    assert np.abs(total[inside]).max() < 0.1
