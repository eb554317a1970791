"""Double layer (gyps_dl_apply) against the oracle: FP64 and DF64 1e-10, FP32 1e-5,
on an ellipsoid and a sphere, Laplace and Helmholtz, several columns."""
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
    return g.Mesh(v, t, q), oracle.Mesh(v, t, q)


@pytest.mark.parametrize("k", [0.0, 6.0])
@pytest.mark.parametrize("nrhs", [1, 3, 6])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("df64", 1e-10), ("fp32", 1e-5)])
def test_dl_apply_vs_oracle(g, pair, k, nrhs, prec, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(nrhs + 3), om.nv, nrhs)
    y = g.dl_apply(gm, k, torch.as_tensor(x).cuda(), prec=prec).cpu().numpy()
    assert rel(y, om.dl_apply(k, x)) < tol


def test_dl_host_buffers_and_errors(g, pair):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(0), om.nv, 2)
    yh = g.dl_apply(gm, 3.0, torch.as_tensor(x), prec="fp64")
    yd = g.dl_apply(gm, 3.0, torch.as_tensor(x).cuda(), prec="fp64").cpu()
    assert not yh.is_cuda and rel(yh.numpy(), yd.numpy()) < 1e-13
    with pytest.raises(g.GypsError) as e:
        g.dl_apply(gm, 3.0, torch.as_tensor(x).cuda(), prec="tc_bf16x3")
    assert e.value.status == "UNSUPPORTED"


def test_dl_gauss_law_on_the_sphere(g):
    """K 1 = -M 1 / 2 on the unit sphere at k = 0, to the oracle's discretisation error."""
    v, t = synth.icosphere(3)
    gm = g.Mesh(v, t, 3)
    om = oracle.Mesh(v, t, 3)
    one = np.ones(om.nv, dtype=complex)
    y = g.dl_apply(gm, 0.0, torch.as_tensor(one).cuda(), prec="fp32").cpu().numpy()
    m1 = om.mass() @ one
    assert np.linalg.norm(y + 0.5 * m1) / np.linalg.norm(m1) < 5e-4
