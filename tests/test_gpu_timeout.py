"""Bounded device waits that run out (the TIMEOUT path), without faulting or
hanging the GPU: gyps_set_wait_polls(0) makes every pipeline wait of the far
kernels give up at once; the kernel records it in the mesh's error word,
drains its copies and products in flight (with the default limit) and returns.
A synchronous apply then returns TIMEOUT, an asynchronous one leaves the word
for gyps_mesh_check, and the next apply with the default limit is correct."""
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
    g.load()
    yield g
    g.set_wait_polls(-1)


@pytest.fixture(scope="module")
def pair(g):
    v, t = synth.icosphere(3)
    return g.Mesh(v, t, 3), oracle.Mesh(v, t, 3)


@pytest.mark.parametrize("prec,nrhs,tol", [("fp32", 2, 1e-5), ("tc_bf16x3", 16, 1e-4)])
def test_wait_runs_out_then_next_apply_is_correct(g, pair, prec, nrhs, tol):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(77), om.nv, nrhs)
    xh = torch.as_tensor(x)  # host buffer: the synchronous path reports its own waits
    g.set_wait_polls(0)
    try:
        with pytest.raises(g.GypsError) as e:
            g.sl_apply(gm, 6.0, xh, prec=prec)
        assert e.value.status == "TIMEOUT"
    finally:
        g.set_wait_polls(-1)
    y = g.sl_apply(gm, 6.0, xh, prec=prec).numpy()
    assert rel(y, om.apply(6.0, x)) < tol


def test_asynchronous_apply_reports_through_mesh_check(g, pair):
    gm, om = pair
    x = torch.as_tensor(synth.random_complex(np.random.default_rng(78), om.nv, 1)).cuda()
    gm.check()  # nothing pending
    g.set_wait_polls(0)
    try:
        g.sl_apply(gm, 6.0, x, prec="fp32")  # device buffers: returns after launching
    finally:
        g.set_wait_polls(-1)
    with pytest.raises(g.GypsError) as e:
        gm.check()
    assert e.value.status == "TIMEOUT"
    gm.check()  # the word was cleared
    y = g.sl_apply(gm, 6.0, x, prec="fp32")
    gm.check()
    assert rel(y.cpu().numpy(), om.apply(6.0, x.cpu().numpy())) < 1e-5


def test_synchronous_call_ignores_an_earlier_asynchronous_failure(g, pair):
    """A failure left in the word by an asynchronous apply is not reported by
    the next synchronous call (it clears the word before its own launches)."""
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(79), om.nv, 1)
    g.set_wait_polls(0)
    try:
        g.sl_apply(gm, 6.0, torch.as_tensor(x).cuda(), prec="fp32")
    finally:
        g.set_wait_polls(-1)
    torch.cuda.synchronize()
    y = g.sl_apply(gm, 6.0, torch.as_tensor(x), prec="fp32").numpy()
    assert rel(y, om.apply(6.0, x)) < 1e-5
    gm.check()


def test_set_wait_polls_rejects_out_of_range(g):
    with pytest.raises(g.GypsError) as e:
        g.set_wait_polls(1 << 31)
    assert e.value.status == "INVALID"
