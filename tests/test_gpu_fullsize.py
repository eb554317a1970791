"""Full-size workloads against the oracle on sampled rows and columns.

batch12_r64: the uneven batch of 12 meshes (icospheres of 320 to 81920
triangles and 7 random ellipsoids, q = 3, k_i ~ U[2, 24], 64 right-hand sides)
in both forms of gyps_batch_apply, the tensor-core applies (tolerance 1e-4)
and the persistent FP32 CUDA-core launch (1e-5); every mesh is checked on
sampled rows for a spread of columns.

assemble_sphere10242: the dense FP32 and FP64 assemblies of the 10242-vertex
sphere (q = 3, k = 16; V is 1.68 GB): sampled columns V e_j against the
oracle's apply to unit vectors, and sampled rows against the oracle's far part
applied to unit vectors (the Gauss-Gauss part is complex symmetric, a property
the oracle pins) plus the rows of its correction C.
"""
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
    return g


@pytest.fixture(scope="module")
def batch_meshes(g):
    items, _ = synth.batch_workload(nrhs=64)
    meshes = [g.Mesh(it["vtx"], it["tri"], 3) for it in items]
    yield items, meshes
    for m in meshes:
        m.close()


@pytest.mark.slow
@pytest.mark.parametrize("cuda_cores", [False, True])
def test_batch12_r64_full_size_sampled_rows(g, batch_meshes, cuda_cores):
    items, meshes = batch_meshes
    b = g.Batch([(m, it["k"]) for m, it in zip(meshes, items)], 64, graph=True, cuda_cores=cuda_cores)
    assert b.info["tensor_cores"] == (0 if cuda_cores else 1)
    xs = []
    for i, m in enumerate(meshes):
        x = synth.random_complex(np.random.default_rng(500 + i), m.nv, 64)
        b.X[i].copy_(torch.as_tensor(x))
        xs.append(x)
    ys = [y.cpu().numpy() for y in b.apply()]
    torch.cuda.synchronize()
    cols = np.arange(0, 64, 9)  # 8 of the 64 columns
    tol = 1e-5 if cuda_cores else 1e-4
    rng = np.random.default_rng(1804)
    for i, it in enumerate(items):
        om = oracle.Mesh(it["vtx"], it["tri"], 3)
        rows = np.sort(rng.choice(om.nv, min(24, om.nv), replace=False))
        ref = om.apply(it["k"], xs[i][:, cols], rows=rows)[rows]
        assert rel(ys[i][rows][:, cols], ref) < tol, (i, it["kind"], it["level"])
    b.close()


@pytest.mark.slow
def test_assemble_sphere10242_sampled_rows_and_columns(g):
    v, t = synth.icosphere(5)
    k = 16.0
    om = oracle.Mesh(v, t, 3)
    gm = g.Mesh(v, t, 3)
    nv = om.nv
    rng = np.random.default_rng(10242)
    cols = np.sort(rng.choice(nv, 6, replace=False))
    rows = np.sort(rng.choice(nv, 6, replace=False))
    e_cols = np.zeros((nv, len(cols)), dtype=np.complex128)
    e_cols[cols, np.arange(len(cols))] = 1.0
    e_rows = np.zeros((nv, len(rows)), dtype=np.complex128)
    e_rows[rows, np.arange(len(rows))] = 1.0
    ref_cols = om.apply(k, e_cols)                       # V e_j
    ref_rows = om.far_apply(k, e_rows).T + om.near.tocsr()[rows].toarray()  # e_i^T V
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-10)):
        V = g.sl_assemble(gm, k, prec=prec)
        got_cols = V[:, torch.as_tensor(cols, device=V.device)].cpu().numpy()
        got_rows = V[torch.as_tensor(rows, device=V.device), :].cpu().numpy()
        del V
        torch.cuda.empty_cache()
        assert rel(got_cols, ref_cols) < tol, prec
        assert rel(got_rows.T, ref_rows.T) < tol, prec
    gm.close()
