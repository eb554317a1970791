"""Pins of the compressed far field of the oracle (Sec. 5.3: blocks of far-apart
clusters replaced by low-rank approximations to a tolerance).

The adaptive cross approximation recovers an exactly low-rank matrix, cannot
beat the truncated SVD's rank on a real block, and meets its tolerance; the
blocks are exact submatrices of the dense far part and cover every entry once;
the compressed apply approaches the dense apply as the tolerance shrinks and
equals it when no block is admissible."""
import numpy as np
import pytest

import oracle
import synth
from oracle import hmat


@pytest.fixture(scope="module")
def sphere3():
    v, t = synth.icosphere(3)
    return oracle.Mesh(v, t, 3)


@pytest.fixture(scope="module")
def vfar3(sphere3):
    return sphere3.assemble_far(8.0)


def test_aca_recovers_an_exactly_low_rank_matrix():
    rng = np.random.default_rng(0)
    a = (rng.normal(size=(90, 6)) + 1j * rng.normal(size=(90, 6))) @ (
        rng.normal(size=(6, 70)) + 1j * rng.normal(size=(6, 70)))
    U, W = hmat.aca(a, 1e-12)
    assert U.shape[1] <= 8
    assert np.linalg.norm(a - U @ W.T) <= 1e-11 * np.linalg.norm(a)


def test_clusters_partition_and_blocks_are_exact_submatrices(sphere3, vfar3):
    cf = hmat.CompressedFar(sphere3, 8.0, eps=1e-4, leaf=16, eta=1.0, vfar=vfar3)
    seen = np.concatenate(cf.clusters)
    assert np.array_equal(np.sort(seen), np.arange(sphere3.nv))
    cover = np.zeros((sphere3.nv, sphere3.nv), dtype=np.int64)
    for s, t, _, _ in cf.blocks:
        cover[np.ix_(cf.clusters[s], cf.clusters[t])] += 1
    assert (cover == 1).all()
    vf = vfar3
    for s, t in ((0, 0), (0, 40), (37, 3)):
        b = cf.block(s, t)
        ref = vf[np.ix_(cf.clusters[s], cf.clusters[t])]
        assert np.abs(b - ref).max() <= 1e-13 * np.abs(ref).max()


def test_aca_meets_its_tolerance_and_not_below_the_svd_rank(sphere3, vfar3):
    cf = hmat.CompressedFar(sphere3, 8.0, eps=1e-4, leaf=16, eta=1.0, vfar=vfar3)
    lowrank = [(s, t, d) for s, t, kind, d in cf.blocks if kind == "lowrank"]
    assert len(lowrank) > 20
    for s, t, (U, W) in lowrank[::7]:
        a = vfar3[np.ix_(cf.clusters[s], cf.clusters[t])]
        err = np.linalg.norm(a - U @ W.T) / np.linalg.norm(a)
        assert err < 1e-3, err
        sv = np.linalg.svd(a, compute_uv=False)
        tail = np.sqrt(np.cumsum((sv ** 2)[::-1])[::-1])  # tail[r] = |A - A_r|_F
        svd_rank = int(np.argmax(tail <= err * np.linalg.norm(a)))
        assert U.shape[1] >= svd_rank


def test_compressed_apply_converges_to_the_dense_apply(sphere3, vfar3):
    x = synth.random_complex(np.random.default_rng(3), sphere3.nv, 2)
    ref = sphere3.far_apply(8.0, x)
    errs = []
    for eps in (1e-2, 1e-4, 1e-6):
        cf = hmat.CompressedFar(sphere3, 8.0, eps=eps, leaf=16, eta=1.0, vfar=vfar3)
        y = cf.apply(x)
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-3 and errs[2] < 1e-5
    exact = hmat.CompressedFar(sphere3, 8.0, eps=1e-4, leaf=16, eta=1e9, vfar=vfar3)
    assert all(kind == "dense" for _, _, kind, _ in exact.blocks)
    assert np.linalg.norm(exact.apply(x) - ref) <= 1e-12 * np.linalg.norm(ref)
