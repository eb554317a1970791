"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test would fail for a plausible mistake in the oracle: a wrong quadrature
point or weight, a dropped or misplaced 1/(4 pi), a wrong sign in exp(ikr), a
transposed correction block, a missing self-pair term, a wrong vertex index.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.quadrature_ref import inner_integral, monomial_integral

SKEW = [np.array([0.1, -0.2, 0.3]), np.array([1.3, 0.1, -0.2]), np.array([0.4, 0.9, 0.5])]


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("q,degree", [(1, 1), (3, 2), (7, 5)])
def test_quadrature_exact_on_monomials(q, degree):
    """dom(mesh, q) (Sec. 4.2): the q-point rule integrates all barycentric
    monomials up to its degree exactly on a skewed triangle, and misses one of
    the next degree."""
    bary, w = oracle.quad_rule(q)
    assert abs(w.sum() - 1.0) < 1e-15
    vtx = np.array(SKEW)
    x, wk = oracle.quad_points(vtx, np.array([[0, 1, 2]], dtype=np.int32), q)
    area = oracle.triangle_areas(vtx, np.array([[0, 1, 2]]))[0]
    # the points are the barycentric combinations of the vertices
    assert np.allclose(x, bary @ vtx, atol=1e-15)
    worst_next = 0.0
    for a in range(degree + 2):
        for b in range(degree + 2 - a):
            for c in range(degree + 2 - a - b):
                num = np.sum(wk * bary[:, 0] ** a * bary[:, 1] ** b * bary[:, 2] ** c)
                ref = monomial_integral(area, a, b, c)
                if a + b + c <= degree:
                    assert abs(num - ref) <= 1e-15 * max(1.0, abs(ref)) * 10
                else:
                    worst_next = max(worst_next, abs(num - ref))
    assert worst_next > 1e-6


def test_mass_matrix_closed_form():
    """Eq. (A=BWB) is an equality when the rule is exact: Phi^T W Phi equals the
    P1 element mass matrix area/12 (1 + delta_ij) assembled over triangles."""
    v, t = synth.icosphere(1)
    areas = oracle.triangle_areas(v, t)
    ref = np.zeros((v.shape[0], v.shape[0]))
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    for tt, a in zip(t, areas):
        ref[np.ix_(tt, tt)] += a * loc
    for q in (3, 7):
        m = oracle.mass_matrix(v, t, q).toarray()
        assert np.abs(m - ref).max() < 1e-15 * 20
    # the centroid rule is not exact for the mass matrix
    assert np.abs(oracle.mass_matrix(v, t, 1).toarray() - ref).max() > 1e-4


# ---------------------------------------------------- closed-form 1/r integral
@pytest.mark.parametrize(
    "x",
    [
        [0.6, 0.35, 0.2],      # inside, projected
        [0.55, 0.3, 0.2],
        [0.6, 0.4, 0.2 + 1e-3],  # off-plane, close
        [3.0, 2.0, -1.5],      # far
        [-0.5, -0.5, 0.0],     # off the triangle, distance measured along the plane normal
    ],
)
def test_p1_inv_r_vs_duffy(x):
    """Sec. 5.2: the y-integral of lambda_j/|x - y| done analytically equals a
    high-order Duffy/polar quadrature of the same integral."""
    x = np.asarray(x, dtype=np.float64)
    ex = oracle.p1_inv_r(x, *SKEW)
    num = inner_integral(x, SKEW, lambda r: 1.0 / r, ng=80)
    assert np.abs(ex - num).max() < 1e-12 * max(1.0, np.abs(num).max())


def test_p1_inv_r_in_plane_points():
    """Points in the plane of the triangle (d = 0): interior points, a point on
    an edge's extension and an exterior point."""
    P = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.2, 0.9, 0.0])]
    for x in ([0.3, 0.3, 0.0], [0.7, 0.05, 0.0], [1.5, 0.0, 0.0], [1.5, -0.5, 0.0], [-0.4, 0.6, 0.0]):
        x = np.asarray(x, dtype=np.float64)
        ex = oracle.p1_inv_r(x, *P)
        num = inner_integral(x, P, lambda r: 1.0 / r, ng=160)  # thin sub-triangles near an edge
        assert np.abs(ex - num).max() < 1e-12, (x, ex, num)


def test_p1_inv_r_vertex_closed_form():
    """At a vertex of a right isosceles triangle with legs h, int_T 1/|x - y|
    equals sqrt(2) h ln(1 + sqrt 2): in polar coordinates about the right-angle
    vertex it is int_0^{pi/2} h / (cos t + sin t) dt."""
    h = 0.7
    P = [np.array([0.0, 0.0, 0.0]), np.array([h, 0.0, 0.0]), np.array([0.0, h, 0.0])]
    x = np.array([0.0, 0.0, 0.0])
    ex = oracle.p1_inv_r(x, *P)
    assert abs(ex.sum() - np.sqrt(2.0) * h * np.log(1.0 + np.sqrt(2.0))) < 1e-14


def test_p1_inv_r_far_field():
    """Far away, int_T lambda_j/|x - y| -> area/(3 |x - c|) (c: centroid)."""
    c = sum(SKEW) / 3.0
    area = 0.5 * np.linalg.norm(np.cross(SKEW[1] - SKEW[0], SKEW[2] - SKEW[0]))
    for dist in (1e3, 1e4):
        x = c + dist * np.array([0.3, -0.5, 0.81])
        x = c + dist * (x - c) / np.linalg.norm(x - c)
        ex = oracle.p1_inv_r(x, *SKEW)
        assert np.abs(ex - area / (3.0 * dist)).max() < 1e-3 * area / (3.0 * dist) * (1e3 / dist) * 10


# ------------------------------------------------------------- correction C
def test_near_pairs_share_a_vertex():
    """Near set = ordered pairs of triangles with a common vertex (a == b included)."""
    v, t = synth.icosphere(1)
    pa, pb = oracle.near_pairs(t, v.shape[0])
    got = set(zip(pa.tolist(), pb.tolist()))
    ref = set()
    for a in range(t.shape[0]):
        for b in range(t.shape[0]):
            if set(t[a].tolist()) & set(t[b].tolist()):
                ref.add((a, b))
    assert got == ref
    # icosphere: 5-valent or 6-valent vertices, 13 neighbours (incl. itself) for regular ones
    counts = np.bincount(pa)
    assert counts.min() >= 10 and counts.max() <= 13


@pytest.mark.parametrize("q", [1, 3])
def test_near_blocks_vs_brute_force(q):
    """Sec. 5.2 correction, element by element on a curved mesh: the analytic
    y-integral replaced by an independent Duffy quadrature; the Gauss sum
    skips only the point paired with itself; row index = test vertex of a."""
    v, t = synth.icosphere(0)
    pa, pb = oracle.near_pairs(t, v.shape[0])
    sel = np.arange(0, pa.shape[0], 7)
    pa, pb = pa[sel], pb[sel]
    blk = oracle.near_blocks(v, t, q, pa, pb)
    bary, wr = oracle.quad_rule(q)
    areas = oracle.triangle_areas(v, t)
    for p in range(pa.shape[0]):
        a, b = pa[p], pb[p]
        A = v[t[a]]
        B = v[t[b]]
        ref = np.zeros((3, 3))
        for kq in range(q):
            xk = bary[kq] @ A
            ex = inner_integral(xk, B, lambda r: 1.0 / r, ng=60)
            gs = np.zeros(3)
            for lq in range(q):
                if a == b and lq == kq:
                    continue
                yl = bary[lq] @ B
                gs += wr[lq] * areas[b] * bary[lq] / np.linalg.norm(xk - yl)
            ref += wr[kq] * areas[a] * np.outer(bary[kq], ex - gs) / (4 * np.pi)
        assert np.abs(blk[p] - ref).max() < 1e-12, (a, b)


def test_coincident_block_vs_brute_force_helmholtz():
    """One flat triangle, V's 3x3 block = far part (with G_kk = ik) + C.
    Against outer Gauss x inner Duffy quadrature of exp(ikr)/r the error is the
    Gauss error of the smooth remainder, O(h^2); leaving out the self pair's
    i k term would leave an O(h) error."""
    k = 3.0
    errs = []
    for h in (0.1, 0.05):
        P = [np.array([0.0, 0.0, 0.0]), np.array([h, 0.0, 0.0]), np.array([0.3 * h, 0.8 * h, 0.0])]
        m = oracle.Mesh(np.array(P), np.array([[0, 1, 2]], dtype=np.int32), 7)
        V = m.assemble(k)
        bary, _ = oracle.quad_rule(7)
        ref = np.zeros((3, 3), dtype=complex)
        for kk in range(7):
            inner = inner_integral(m.x[kk], P, lambda r: np.exp(1j * k * r) / r, ng=60)
            ref += m.w[kk] * np.outer(bary[kk], inner) / (4 * np.pi)
        errs.append(np.abs(V - ref).max() / np.abs(ref).max())
    assert errs[1] < 5e-5
    assert errs[0] / errs[1] > 3.5


@pytest.mark.parametrize("shared", ["edge", "vertex"])
def test_adjacent_pair_vs_brute_force_helmholtz(shared):
    """Two triangles that share an edge (or a vertex), slightly out of plane:
    the whole 4x4 (5x5) V, far part with the correction, against the same outer
    Gauss rule with the inner integrals of exp(ikr)/r by Duffy quadrature over
    each triangle.  The difference is the Gauss error of the smooth remainder
    (exp(ikr) - 1)/r, O(h^2); a wrong sign, a transposed block or a dropped
    correction between neighbours leaves an O(1) or O(h) error."""
    k = 4.0
    errs = []
    for h in (0.1, 0.05):
        P = np.array([[0.0, 0.0, 0.0], [h, 0.0, 0.0], [0.4 * h, 0.9 * h, 0.0], [0.6 * h, -0.8 * h, 0.15 * h],
                      [-0.7 * h, -0.2 * h, 0.1 * h], [-0.3 * h, -0.9 * h, -0.05 * h]])
        if shared == "edge":
            tri = np.array([[0, 1, 2], [1, 0, 3]], dtype=np.int32)
        else:
            tri = np.array([[0, 1, 2], [0, 4, 5]], dtype=np.int32)
        used = np.unique(tri)
        remap = {int(v): i for i, v in enumerate(used)}
        tri = np.vectorize(remap.get)(tri).astype(np.int32)
        P = P[used]
        m = oracle.Mesh(P, tri, 7)
        V = m.assemble(k)
        bary, _ = oracle.quad_rule(7)
        ref = np.zeros_like(V)
        for a in range(2):
            for b in range(2):
                Pb = [P[v] for v in tri[b]]
                for kk in range(7):
                    xk = m.x[7 * a + kk]
                    inner = inner_integral(xk, Pb, lambda r: np.exp(1j * k * r) / r, ng=60)
                    blk = m.w[7 * a + kk] * np.outer(bary[kk], inner) / (4 * np.pi)
                    ref[np.ix_(tri[a], tri[b])] += blk
        errs.append(np.abs(V - ref).max() / np.abs(ref).max())
    assert errs[1] < 5e-5
    assert errs[0] / errs[1] > 3.5


# ------------------------------------------------------------- far part
def test_far_part_is_complex_symmetric():
    """Eq. (BEM) with the same points and space on both sides: Phi^T W G W Phi
    is complex symmetric (G_kl = G_lk, plain transpose, no conjugation)."""
    v, t = synth.icosphere(2)
    m = oracle.Mesh(v, t, 3)
    vf = m.assemble_far(4.0)
    assert np.abs(vf - vf.T).max() < 1e-14 * np.abs(vf).max()
    assert np.abs(vf - vf.conj().T).max() > 1e-3 * np.abs(vf).max()


def test_dense_and_matrix_free_agree():
    v, t = synth.icosphere(2)
    m = oracle.Mesh(v, t, 3)
    rng = np.random.default_rng(0)
    x = synth.random_complex(rng, m.nv, 2)
    y = m.apply(5.0, x)
    y2 = m.assemble(5.0) @ x
    assert np.abs(y - y2).max() < 1e-13 * np.abs(y).max()
    rows = np.array([0, 7, 100, 161])
    y3 = m.apply(5.0, x, rows=rows)
    assert np.abs(y3[rows] - y[rows]).max() < 1e-14 * np.abs(y).max()


# ------------------------------------------------------- sphere closed forms
def _sph_harm_real(n, v):
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    return {0: np.ones_like(x), 1: z, 2: 3 * z * z - 1, 3: x * y * z, 4: x * y * (7 * z * z - 1)}[n]


@pytest.mark.parametrize("k", [0.0, 5.0])
@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_sphere_eigenvalues_converge(k, n):
    """Unit sphere: S Y_n = mu_n Y_n with mu_n = 1/(2n+1) (k = 0) and
    i k j_n(k) h_n(k) (k > 0).  With u the P1 interpolant of Y_n,
    ||V u - mu_n M u|| / ||mu_n M u|| -> 0 at rate ~h^2 (x4 per level)."""
    mu = oracle.sphere_eigenvalue(n, k)
    errs = []
    for level in (1, 2, 3):
        v, t = synth.icosphere(level)
        m = oracle.Mesh(v, t, 3)
        u = _sph_harm_real(n, v)
        ref = mu * (m.mass() @ u)
        errs.append(np.linalg.norm(m.apply(k, u) - ref) / np.linalg.norm(ref))
    assert errs[-1] < (0.02 if k == 0.0 else 0.08), errs
    assert errs[1] / errs[2] > 3.0 and errs[0] / errs[1] > 2.5, errs


def test_rhs_constant_wave_is_mass_row_sum():
    """Sec. 5.4 right-hand side with k = 0: F_i = int phi_i = sum of area/3 over
    the triangles at vertex i."""
    v, t = synth.icosphere(2)
    m = oracle.Mesh(v, t, 3)
    f = m.rhs_planewave(0.0, [(0.0, 0.0, 1.0)])[:, 0]
    ref = np.zeros(m.nv)
    np.add.at(ref, t.reshape(-1), np.repeat(oracle.triangle_areas(v, t) / 3.0, 3))
    assert np.abs(f - ref).max() < 1e-15 * 10


# ------------------------------------------------------------------ solves
@pytest.mark.slow
def test_gmres_matches_lu_sphere642():
    """Workload sphere642_k5_q3: GMRES (CGS2, Givens) to 1e-12 agrees with the
    direct solve (the paper's LHS \\ RHS) to 1e-10."""
    v, t = synth.icosphere(3)
    m = oracle.Mesh(v, t, 3)
    a = m.assemble(5.0)
    f = m.rhs_planewave(5.0, [(0.0, 0.0, 1.0)])[:, 0]
    x_lu = oracle.solve_lu(a, f)
    x_g, it, res = oracle.gmres(lambda z: a @ z, f, tol=1e-12, restart=100)
    assert res <= 1e-12 * 1.5
    assert np.linalg.norm(x_g - x_lu) / np.linalg.norm(x_lu) < 1e-10
    # restarts give the same answer
    x_r, it_r, res_r = oracle.gmres(lambda z: a @ z, f, tol=1e-12, restart=15)
    assert np.linalg.norm(x_r - x_lu) / np.linalg.norm(x_lu) < 1e-10


def test_mie_series_convergence():
    """Sound-soft sphere (Sec. 5.4): the discrete density of V lambda = F
    converges to the Mie series lambda = sum (2n+1) i^n P_n(d.x)/(i k h_n(k))
    (mass-weighted relative L2 error), halving at least per refinement."""
    k = 3.0
    d = np.array([0.0, 0.0, 1.0])
    errs = []
    for level in (1, 2, 3):
        v, t = synth.icosphere(level)
        m = oracle.Mesh(v, t, 3)
        lam = oracle.solve_lu(m.assemble(k), m.rhs_planewave(k, [d])[:, 0])
        ref = oracle.mie_density(k, d, v)
        mm = m.mass()
        e = lam - ref
        errs.append(np.sqrt(np.real(e.conj() @ (mm @ e)) / np.real(ref.conj() @ (mm @ ref))))
    assert errs[-1] < 0.03, errs
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0, errs
    # the opposite propagation direction must not match
    v, t = synth.icosphere(3)
    ref_flip = oracle.mie_density(k, -d, v)
    e = lam - ref_flip
    assert np.sqrt(np.real(e.conj() @ (mm @ e)) / np.real(ref_flip.conj() @ (mm @ ref_flip))) > 0.3


def test_mie_series_is_the_laplace_limit_free():
    """At k -> 0 the plane wave tends to 1 and the density to 1 (S 1 = 1 on the
    unit sphere); the series at small k is close to 1 + O(k)."""
    lam = oracle.mie_density(1e-3, [0, 0, 1], np.array([[1.0, 0, 0], [0, 0, 1.0]]))
    assert np.abs(lam - 1.0).max() < 1e-2


# ------------------------------------------------------------------ meshes
@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere_counts_and_orientation(level):
    v, t = synth.icosphere(level)
    nv, nt = synth.unit_sphere_counts(level)
    assert v.shape == (nv, 3) and t.shape == (nt, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    assert (np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) > 0).all()
    # closed surface: every edge shared by exactly two triangles
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert (cnt == 2).all()


def _octahedron():
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=float)
    tri = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                t = [sx, sy, sz]
                P = v[t]
                if np.cross(P[1] - P[0], P[2] - P[0]) @ P.mean(0) < 0:
                    t = [sx, sz, sy]
                tri.append(t)
    return v, np.array(tri, dtype=np.int32)


def test_tiny_mesh_approaches_the_exact_galerkin_matrix():
    """Octahedron surface, k = 2: the exact Galerkin V_ij = (1/4pi) int int phi_i phi_j
    exp(ikr)/r by brute force (outer: collapsed 10 x 10 Gauss-Legendre product rule per
    triangle; inner: Duffy quadrature of order 30, which handles the coincident and
    adjacent singularities).  The discrete V (Gauss points, far part with G_kk = ik, the
    '[1/r]' correction) approaches it as the rule grows: about 26 % (q = 1), 7.7 % (q = 3),
    1.1 % (q = 7); the brute force itself is converged to about 1e-3 at a coarser order."""
    v, tri = _octahedron()
    k = 2.0
    g, w = np.polynomial.legendre.leggauss(10)
    g, w = (g + 1) / 2, w / 2
    U, W = np.meshgrid(g, g, indexing="ij")
    WW = np.outer(w, w)
    exact = np.zeros((6, 6), dtype=complex)
    for a in range(len(tri)):
        A, B, C = v[tri[a]]
        X = (A + U[..., None] * (B - A) + (U * W)[..., None] * (C - B)).reshape(-1, 3)
        wx = (np.linalg.norm(np.cross(B - A, C - A)) * U * WW).reshape(-1)
        lam = np.stack([1 - U, U * (1 - W), U * W], -1).reshape(-1, 3)
        for b in range(len(tri)):
            Pb = [v[i] for i in tri[b]]
            for xx, ww, la in zip(X, wx, lam):
                inner = inner_integral(xx, Pb, lambda r: np.exp(1j * k * r) / r, ng=30)
                exact[np.ix_(tri[a], tri[b])] += ww * np.outer(la, inner) / (4 * np.pi)
    errs = []
    for q in (1, 3, 7):
        Vq = oracle.Mesh(v, tri, q).assemble(k)
        errs.append(np.abs(Vq - exact).max() / np.abs(exact).max())
    assert errs[2] < 2e-2 and errs[1] > 3 * errs[2] and errs[0] > 2 * errs[1], errs
