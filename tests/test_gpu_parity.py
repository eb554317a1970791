"""GPU path (through the C ABI) against the FP64 oracle on identical inputs.

Tolerances (relative, per right-hand-side column; parity.rel bounds the
column's 2-norm error and every element's error against the column's largest
entry): FP64 paths 1e-10; FP32 far kernel 1e-5 (FP32 kernel values and
compensated FP32 sums; the near correction stays FP64).
Sizes span several source tiles of 256 points and a ragged tail; k = 64 puts
the phases k r up to about 130 rad (the wavenumber of the 163842-vertex
sphere workload).
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


def to_np(t):
    return t.detach().cpu().numpy()


MESHES = {
    "ico2_q3": lambda: (*synth.icosphere(2), 3),
    "ico3_q7": lambda: (*synth.icosphere(3), 7),
    "ell2_q1": lambda: (*synth.ellipsoid(2, (0.6, 1.3, 1.9), (1.0, 2.0, 0.5), 0.7), 1),
}


@pytest.fixture(scope="module", params=sorted(MESHES))
def pair(request, g):
    v, t, q = MESHES[request.param]()
    return g.Mesh(v, t, q), oracle.Mesh(v, t, q)


def test_quadrature_points(pair):
    gm, om = pair
    xw = to_np(gm.quad_points())
    assert np.abs(xw[:, :3] - om.x).max() < 1e-15 * 8
    assert np.abs(xw[:, 3] - om.w).max() <= 1e-16 * 8 * om.w.max()


def test_near_matrix_pattern_and_values(pair):
    gm, om = pair
    rowptr, col, val = gm.near_csr()
    c = om.near.tocsr()
    c.sort_indices()
    assert np.array_equal(rowptr, c.indptr.astype(np.int64))
    assert np.array_equal(col, c.indices.astype(np.int32))
    assert np.abs(val - c.data).max() <= 1e-12 * np.abs(c.data).max()


@pytest.mark.parametrize("k", [0.0, 5.0, 16.0])
@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_apply_fp64(pair, g, k, nrhs):
    gm, om = pair
    rng = np.random.default_rng(11 + nrhs)
    x = synth.random_complex(rng, om.nv, nrhs)
    y = g.sl_apply(gm, k, torch.as_tensor(x).cuda(), prec="fp64")
    assert rel(to_np(y), om.apply(k, x)) < 1e-10


@pytest.mark.parametrize("k", [0.0, 5.0, 16.0, 64.0])
@pytest.mark.parametrize("nrhs", [1, 3, 6, 11])
def test_apply_df64(pair, g, k, nrhs):
    """Double-float products: FP64-class accuracy against the oracle and within
    1e-11 of the FP64 GPU form (k = 64 puts phases k r up to about 130 rad)."""
    gm, om = pair
    rng = np.random.default_rng(31 + nrhs)
    x = synth.random_complex(rng, om.nv, nrhs)
    xd = torch.as_tensor(x).cuda()
    y = to_np(g.sl_apply(gm, k, xd, prec="df64"))
    assert rel(y, om.apply(k, x)) < 1e-10
    assert rel(y, to_np(g.sl_apply(gm, k, xd, prec="fp64"))) < 1e-11


@pytest.mark.parametrize("k", [0.0, 5.0, 16.0, 64.0])
@pytest.mark.parametrize("nrhs", [1, 2, 5, 13])
def test_apply_fp32(pair, g, k, nrhs):
    gm, om = pair
    rng = np.random.default_rng(23 + nrhs)
    x = synth.random_complex(rng, om.nv, nrhs)
    y = g.sl_apply(gm, k, torch.as_tensor(x).cuda(), prec="fp32")
    assert rel(to_np(y), om.apply(k, x)) < 1e-5


@pytest.mark.parametrize("k", [7.0, 64.0])
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_far_part_only(pair, g, prec, k):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(5), om.nv, 2)
    y = g.sl_apply(gm, k, torch.as_tensor(x).cuda(), prec=prec, near=False)
    assert rel(to_np(y), om.far_apply(k, x)) < (1e-5 if prec == "fp32" else 1e-10)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_triangle_ranges_add_up(pair, g, prec):
    """Applies over a partition of the test triangles sum to the full apply."""
    gm, om = pair
    x = torch.as_tensor(synth.random_complex(np.random.default_rng(9), om.nv, 3)).cuda()
    full = to_np(g.sl_apply(gm, 4.0, x, prec=prec))
    cuts = [0, om.nt // 3, om.nt // 3 + 1, om.nt]
    parts = sum(to_np(g.sl_apply(gm, 4.0, x, prec=prec, tri_range=(a, b))) for a, b in zip(cuts[:-1], cuts[1:]))
    assert rel(parts, full) < (1e-6 if prec == "fp32" else 1e-12)
    empty = to_np(g.sl_apply(gm, 4.0, x, prec=prec, tri_range=(5, 5)))
    assert np.abs(empty).max() == 0.0


def test_near_correct(pair, g):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(3), om.nv, 2)
    y0 = synth.random_complex(np.random.default_rng(4), om.nv, 2)
    y = torch.as_tensor(y0).cuda().t().contiguous().t()
    g.near_correct(gm, torch.as_tensor(x).cuda(), y)
    assert rel(to_np(y), y0 + om.near @ x) < 1e-13


def test_rhs_planewave(pair, g):
    gm, om = pair
    dirs = synth.plane_wave_dirs(np.random.default_rng(2), 3)
    f = g.rhs_planewave(gm, 6.0, dirs)
    assert rel(to_np(f), om.rhs_planewave(6.0, dirs)) < 1e-13


def test_host_buffers_match_device(pair, g):
    gm, om = pair
    x = synth.random_complex(np.random.default_rng(8), om.nv, 2)
    yd = to_np(g.sl_apply(gm, 3.0, torch.as_tensor(x).cuda(), prec="fp32"))
    yh = g.sl_apply(gm, 3.0, torch.as_tensor(x), prec="fp32").numpy()
    assert rel(yh, yd) < 1e-12


def test_dense_assembly_sphere642(g):
    """Workload sphere642_k5_q3: dense 642 x 642 FP64 assembly incl. correction."""
    v, t = synth.icosphere(3)
    om = oracle.Mesh(v, t, 3)
    gm = g.Mesh(v, t, 3)
    for k in (5.0, 0.0):
        ref = om.assemble(k)
        got = to_np(g.sl_assemble(gm, k, prec="fp64"))
        assert rel(got, ref) < 1e-12
        got32 = to_np(g.sl_assemble(gm, k, prec="fp32"))
        assert rel(got32, ref) < 1e-5


@pytest.mark.parametrize("q", [1, 7])
def test_dense_assembly_other_rules(g, q):
    """Dense assembly with the 1- and 7-point rules (both kernels: FP64 triangle
    pairs, FP32 vertex x triangle) on a 320-triangle ellipsoid."""
    v, t = synth.ellipsoid(2, (0.8, 1.2, 1.5), (0.3, 1.0, -0.4), 0.7)
    om = oracle.Mesh(v, t, q)
    gm = g.Mesh(v, t, q)
    ref = om.assemble(7.0)
    got = to_np(g.sl_assemble(gm, 7.0, prec="fp64"))
    assert rel(got, ref) < 1e-12
    got32 = to_np(g.sl_assemble(gm, 7.0, prec="fp32"))
    assert rel(got32, ref) < 1e-5


def test_gmres_sphere642_matches_lu(g):
    """Workload sphere642_k5_q3: FP64 GMRES against the oracle's LU solve.  A
    residual tol bounds the solution error by cond(V) tol, so the LU comparison
    runs at tol 1e-12; the 1e-8 solves are judged by their residual against the
    oracle's dense V and F."""
    v, t = synth.icosphere(3)
    om = oracle.Mesh(v, t, 3)
    gm = g.Mesh(v, t, 3)
    d = [(0.0, 0.0, 1.0)]
    a = om.assemble(5.0)
    fo = om.rhs_planewave(5.0, d)[:, 0]
    ref = oracle.solve_lu(a, fo)
    f = g.rhs_planewave(gm, 5.0, d)
    x, rep = g.gmres_solve(gm, 5.0, f, tol=1e-12, restart=200, prec="fp64", check_prec="fp64")
    assert rep.status == "OK" and rep.true_residual[0] <= 1e-12
    assert np.linalg.norm(to_np(x)[:, 0] - ref) / np.linalg.norm(ref) < 1e-9
    for prec, check in (("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "df64")):
        x8, rep8 = g.gmres_solve(gm, 5.0, f, tol=1e-8, restart=200, prec=prec, check_prec=check, max_refine=5)
        assert rep8.status == "OK" and rep8.true_residual[0] <= 1e-8
        xo = to_np(x8)[:, 0]
        assert np.linalg.norm(a @ xo - fo) / np.linalg.norm(fo) < 1.01e-8


def test_tiny_meshes_and_ragged_tails(g):
    """One triangle (3 points, one partial source tile) and a tetrahedron."""
    v = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.1], [0.1, 0.25, 0.0], [0.1, 0.1, 0.3]])
    for tri in (np.array([[0, 1, 2]], dtype=np.int32), np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [2, 0, 3]], dtype=np.int32)):
        nv = int(tri.max()) + 1
        for q in (1, 3, 7):
            om = oracle.Mesh(v[:nv], tri, q)
            gm = g.Mesh(v[:nv], tri, q)
            x = synth.random_complex(np.random.default_rng(q), nv, 2)
            for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5)):
                y = to_np(g.sl_apply(gm, 2.0, torch.as_tensor(x).cuda(), prec=prec))
                assert rel(y, om.apply(2.0, x)) < tol
            # tensor-core form: one target tile and one source chunk, mostly padding
            x16 = synth.random_complex(np.random.default_rng(10 + q), nv, 16)
            y16 = to_np(g.sl_apply(gm, 2.0, torch.as_tensor(x16).cuda(), prec="tc_bf16x3"))
            assert rel(y16, om.apply(2.0, x16)) < 1e-4


def test_invalid_inputs(g):
    v, t = synth.icosphere(1)
    bad = t.copy()
    bad[3, 1] = v.shape[0]
    with pytest.raises(g.GypsError) as e:
        g.Mesh(v, bad, 3)
    assert e.value.status == "INVALID"
    deg = t.copy()
    deg[0, 1] = deg[0, 0]
    with pytest.raises(g.GypsError):
        g.Mesh(v, deg, 3)
    gm = g.Mesh(v, t, 3)
    x = torch.zeros((gm.nv, 1), dtype=torch.complex128, device="cuda")
    for kbad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(g.GypsError):
            g.sl_apply(gm, kbad, x)
    with pytest.raises(g.GypsError):
        g.sl_apply(gm, 1.0, x, tri_range=(0, gm.nt + 1))
    with pytest.raises(g.GypsError) as e:
        g.sl_apply(gm, 1.0, x, prec="tc_bf16x3")
    assert e.value.status == "UNSUPPORTED"


@pytest.mark.slow
def test_sphere10242_k16_q7_sampled_rows(g):
    """Workload sphere10242_k16_q7 at full size, launch configuration of the
    benchmark: FP32 apply vs the oracle on 64 sampled rows; FP64 apply too."""
    v, t = synth.icosphere(5)
    om = oracle.Mesh(v, t, 7)
    gm = g.Mesh(v, t, 7)
    rng = np.random.default_rng(1804)
    x = synth.random_complex(rng, om.nv, 1)
    rows = np.sort(rng.choice(om.nv, 64, replace=False))
    ref = om.apply(16.0, x, rows=rows)[rows]
    xd = torch.as_tensor(x).cuda()
    y32 = to_np(g.sl_apply(gm, 16.0, xd, prec="fp32"))[rows]
    assert rel(y32, ref) < 1e-5
    y64 = to_np(g.sl_apply(gm, 16.0, xd, prec="fp64"))[rows]
    assert rel(y64, ref) < 1e-10


@pytest.mark.slow
def test_sphere10242_k16_q7_gmres_against_mie(g):
    """Workload sphere10242_k16_q7: sound-soft scattering, FP32 operator in the
    Krylov loop, FP64 true residual <= 1e-6, density close to the Mie series
    (mass-weighted relative L2 error; discretisation error, kh ~ 0.5)."""
    v, t = synth.icosphere(5)
    gm = g.Mesh(v, t, 7)
    d = (1.0, 0.0, 0.0)
    f = g.rhs_planewave(gm, 16.0, [d])
    x, rep = g.gmres_solve(gm, 16.0, f, tol=1e-6, restart=200, maxit=1000, prec="fp32", check_prec="fp64",
                           max_refine=4)
    assert rep.status == "OK" and rep.true_residual[0] <= 1e-6
    lam = to_np(x)[:, 0]
    ref = oracle.mie_density(16.0, d, v)
    mm = oracle.mass_matrix(v, t, 7)
    e = lam - ref
    err = np.sqrt(np.real(e.conj() @ (mm @ e)) / np.real(ref.conj() @ (mm @ ref)))
    assert err < 0.05, err


def test_gmres_wall_clock_limit(g):
    """timeout_ms: a limit that passes before the first inner iteration returns
    TIMEOUT with the report filled and X finite; a generous limit changes nothing."""
    v, t = synth.icosphere(3)
    gm = g.Mesh(v, t, 3)
    F = g.rhs_planewave(gm, 5.0, [[0.0, 0.0, 1.0]])
    x, rep = g.gmres_solve(gm, 5.0, F, tol=1e-12, restart=50, maxit=500, prec="fp32", check_prec="fp64",
                           timeout_ms=1e-6)
    assert rep.status == "TIMEOUT" and rep.iterations <= 1 and not rep.converged.any()
    assert torch.isfinite(torch.view_as_real(x)).all() and np.isfinite(rep.true_residual).all()
    with pytest.raises(g.GypsError) as e:
        g.gmres_solve(gm, 5.0, F, tol=1e-12, prec="fp32", timeout_ms=1e-6, raise_on_fail=True)
    assert e.value.status == "TIMEOUT"
    x2, rep2 = g.gmres_solve(gm, 5.0, F, tol=1e-8, restart=200, maxit=500, prec="fp32", check_prec="fp64",
                             timeout_ms=6e5)
    assert rep2.status == "OK" and rep2.converged.all()
    with pytest.raises(g.GypsError) as e:
        g.gmres_solve(gm, 5.0, F, timeout_ms=-1.0)
    assert e.value.status == "INVALID"
