"""Batched apply (one persistent launch over many meshes, CUDA graph) against
per-mesh applies and the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle
import synth
from parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def small_batch():
    rng = np.random.default_rng(77)
    specs = [(synth.icosphere(1), 3, 3.0), (synth.ellipsoid(2, (0.7, 1.2, 1.6), (1, 1, 0), 0.4), 7, 0.0),
             (synth.icosphere(2), 1, 7.5), (synth.random_ellipsoid(rng, 1)[:2], 3, 12.0)]
    return [(v, t, q, k) for (v, t), q, k in specs]


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("nrhs", [1, 6, 8])
def test_batch_matches_single_applies_and_oracle(graph, nrhs):
    import paper_1804_00995_gb300 as g
    specs = small_batch()
    meshes = [g.Mesh(v, t, q) for v, t, q, _ in specs]
    b = g.Batch([(m, k) for m, (_, _, _, k) in zip(meshes, specs)], nrhs, graph=graph)
    assert b.info["uses_graph"] == int(graph) and b.info["nmesh"] == len(specs)
    for rep in range(2):  # refill X in place and replay
        xs = []
        for i, m in enumerate(meshes):
            x = synth.random_complex(np.random.default_rng(10 * i + rep), m.nv, nrhs)
            b.X[i].copy_(torch.as_tensor(x))
            xs.append(x)
        ys = b.apply()
        torch.cuda.synchronize()
        for i, (m, (v, t, q, k)) in enumerate(zip(meshes, specs)):
            y = ys[i].cpu().numpy()
            y1 = g.sl_apply(m, k, torch.as_tensor(xs[i]).cuda(), prec="fp32").cpu().numpy()
            assert rel(y, y1) < 1e-6
            assert rel(y, oracle.Mesh(v, t, q).apply(k, xs[i])) < 1e-5
    b.close()


def test_batch_autotune_cache(tmp_path, monkeypatch):
    import paper_1804_00995_gb300 as g
    monkeypatch.setenv("GYPS_TUNE_CACHE", str(tmp_path / "tune.json"))
    specs = small_batch()
    meshes = [g.Mesh(v, t, q) for v, t, q, _ in specs]
    items = [(m, k) for m, (_, _, _, k) in zip(meshes, specs)]
    b1 = g.Batch(items, 8, autotune=True)
    assert b1.info["tuned"] == 1
    assert os.path.exists(tmp_path / "tune.json")
    b2 = g.Batch(items, 8)
    assert b2.info["tuned"] == 2
    assert (b2.info["rhs_chunk"], b2.info["targets_per_thread"]) == (b1.info["rhs_chunk"], b1.info["targets_per_thread"])
    b1.close()
    b2.close()


def test_batch_rejects_host_buffers():
    import ctypes
    import paper_1804_00995_gb300 as g
    v, t = synth.icosphere(1)
    m = g.Mesh(v, t, 3)
    xh = np.zeros(m.nv, dtype=np.complex128)
    arr = (g._BatchItem * 1)()
    arr[0] = g._BatchItem(m.handle.value, 1.0, xh.ctypes.data, m.nv, xh.ctypes.data, m.nv)
    h = ctypes.c_void_p()
    assert g.load().gyps_batch_create(arr, 1, 1, 0, None, ctypes.byref(h)) == 1


def test_batch_tensor_core_mode():
    """>= 16 right-hand sides and every k > 0: the default form is the
    tensor-core apply of each mesh (tolerance of the split bf16 products)."""
    import paper_1804_00995_gb300 as g
    specs = [s for s in small_batch() if s[3] > 0.0]
    meshes = [g.Mesh(v, t, q) for v, t, q, _ in specs]
    b = g.Batch([(m, k) for m, (_, _, _, k) in zip(meshes, specs)], 16)
    assert b.info["tensor_cores"] == 1
    xs = []
    for i, m in enumerate(meshes):
        x = synth.random_complex(np.random.default_rng(40 + i), m.nv, 16)
        b.X[i].copy_(torch.as_tensor(x))
        xs.append(x)
    ys = b.apply()
    torch.cuda.synchronize()
    for i, (v, t, q, k) in enumerate(specs):
        assert rel(ys[i].cpu().numpy(), oracle.Mesh(v, t, q).apply(k, xs[i])) < 1e-4
    b.close()
