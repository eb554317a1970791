"""Multi-rank design on CPU (gloo, world sizes 2 and 3): the operator is
sharded by test triangles with bench.py's partition (triangle_range); each rank
sums the far part over the target points of its triangles and the correction
over its test triangles; one all-reduce of the nv x nrhs result, in the layout
bench.py reduces (the real view of the column-major block's transpose), gives
the full apply.  The arithmetic is the oracle's; what is tested is the
partition and the exchange step."""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
import synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _partial_apply(om, k, x, tri_begin, tri_end):
    """Contribution of test triangles [tri_begin, tri_end) to V x."""
    q = om.q
    tids = np.arange(tri_begin * q, tri_end * q)
    u = om.w[:, None] * (om.phi @ x)
    v = np.zeros((om.nq, x.shape[1]), dtype=np.complex128)
    if tids.size:
        v[tids] = oracle.kernel_matvec(om.x[tids], tids, om.x, u, k)
    y = (om.phi.T @ (om.w[:, None] * v)) / (4.0 * np.pi)
    pa, pb = oracle.near_pairs(om.tri, om.nv)
    sel = (pa >= tri_begin) & (pa < tri_end)
    blk = oracle.near_blocks(om.vtx, om.tri, q, pa[sel], pb[sel])
    for bmat, a, b in zip(blk, pa[sel], pb[sel]):
        ia, ib = om.tri[a], om.tri[b]
        y[ia] += bmat @ x[ib]
    return y


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v, t = synth.icosphere(2)
    om = oracle.Mesh(v, t, 3)
    x = synth.random_complex(np.random.default_rng(1), om.nv, 2)
    tb, te = bench.triangle_range(rank, world, om.nt)
    y = _partial_apply(om, 6.0, x, tb, te)
    yt = torch.as_tensor(np.ascontiguousarray(y.T))  # (nrhs, nv): the transpose of the column-major block
    dist.all_reduce(torch.view_as_real(yt), op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out, yt.numpy().T)
    dist.barrier()
    dist.destroy_process_group()


def test_triangle_ranges_partition():
    for world in (1, 2, 3, 8):
        r = [bench.triangle_range(q, world, 20480) for q in range(world)]
        assert r[0][0] == 0 and r[-1][1] == 20480
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))


@pytest.mark.parametrize("world", [2, 3])
def test_rank_partition_all_reduce(tmp_path, world):
    oracle.build()  # compile once before the ranks start
    import torch.multiprocessing as mp
    out = str(tmp_path / "y.npy")
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    y = np.load(out)
    v, t = synth.icosphere(2)
    om = oracle.Mesh(v, t, 3)
    x = synth.random_complex(np.random.default_rng(1), om.nv, 2)
    ref = om.apply(6.0, x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
