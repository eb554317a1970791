"""Multi-rank design on CPU (gloo, world size 2): the operator is sharded by
test triangles; each rank sums the far part over the target points of its
triangles and the correction over its test triangles; one all-reduce of the
nv x nrhs result gives the full apply.  The arithmetic is the oracle's; what
is tested is the partition and the exchange step."""
import os
import socket

import numpy as np
import pytest

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
    cuts = np.linspace(0, om.nt, world + 1).astype(int)
    y = _partial_apply(om, 6.0, x, cuts[rank], cuts[rank + 1])
    buf = torch.as_tensor(np.stack([y.real, y.imag]))
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out, buf.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partition_all_reduce(tmp_path):
    oracle.build()  # compile once before the ranks start
    import torch.multiprocessing as mp
    out = str(tmp_path / "y.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    v, t = synth.icosphere(2)
    om = oracle.Mesh(v, t, 3)
    x = synth.random_complex(np.random.default_rng(1), om.nv, 2)
    ref = om.apply(6.0, x)
    y = got[0] + 1j * got[1]
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
