"""FP64 CPU oracle of the Galerkin Helmholtz single-layer operator (test infrastructure).

This package is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path in ``paper_1804_00995_gb300``; the only common inputs come from
``synth`` (meshes, directions), which holds none of the operator's arithmetic.

It follows the paper's formulation step by step:

* Sec. 3, Eqs. (approxA), (WB), (A=BWB): quadrature points ``x_k``, weights
  ``w_k``, the sparse basis matrix ``Phi_kj = phi_j(x_k)`` and ``A = Phi^T W Phi``.
* Sec. 5, Eq. (BEM): ``V ~ (1/4pi) Phi^T W_x G W_y Phi`` with
  ``G_kl = exp(ik|x_k - y_l|)/|x_k - y_l|`` evaluated on point clouds.
* Sec. 5.2 (regularize ... '[1/r]'): a sparse correction on pairs of triangles
  sharing a vertex, analytic integral in y minus the Gauss sum, outer Gauss in x.
* Sec. 5.4, Eqs. (Singlelayer), (Singlelayerwf): right-hand side
  ``F_i = int phi_i exp(ik d.x)`` and the solve ``V lambda = F``.
* Sec. 5.4 (radiation operator): the single-layer potential at points, with the
  same '[1/r]' regularisation for triangles near a point.
* Sec. 5.2 with the grady[exp(ikr)/r] kernel: the double layer ``K``, its
  'grady[1/r]' correction in closed form (solid angle and edge logarithms).
* The Brakhage-Werner combined operator ``1/2 M + K - i eta V`` (Brakhage and
  Werner 1965), assembled from the operators above, and its sphere closed form.
* The adjoint double layer ``K'`` (normal at the test point) and the direct
  combined-field operator ``1/2 M + K' - i eta V`` whose solution is the density of
  the paper's sound-soft problem.
* The EFIE of the electromagnetic listing of Sec. 5.5 with RWG functions:
  the vector and divergence parts of ``T`` through the same kernel, their
  '[1/r]' corrections from the P1 closed form, and the Mie amplitudes of the
  perfectly conducting sphere.
* Its MFIE part ``nxK`` (kernel grad_y exp(ikr)/r, 'grady[1/r]' correction from
  the closed form of int lambda (x - y)/R^3) and the combined LHS / RHS of the
  listing, -beta T + (1 - beta)(Id/2 - nxK).

Readings where the paper is silent (all listed with the design notes): the
3-point rule is the interior (2/3, 1/6, 1/6) rule; "close enough" means sharing
at least one vertex; a quadrature point paired with itself gets the kernel's
smooth limit ``i k`` and is left out of the correction's Gauss sum; the outer
rule of the correction is the domain's own rule.

Parity unpinned: the absolute accuracy of the paper's regularisation itself
(the paper prints no values); it is bounded by the sphere convergence checks
and by the comparison with brute-force exact Galerkin entries on a tiny mesh.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gyps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle's C part with gcc (FP64, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.or_quad_rule.argtypes = [ctypes.c_int, dp, dp]
            lib.or_kernel_matvec.argtypes = [ctypes.c_int64, dp, i64p, ctypes.c_int64, dp,
                                             ctypes.c_double, ctypes.c_int64, dp, dp]
            lib.or_kernel_matrix.argtypes = [ctypes.c_int64, dp, i64p, ctypes.c_int64, dp,
                                             ctypes.c_double, dp]
            lib.or_p1_inv_r.argtypes = [dp, dp, dp, dp, dp]
            lib.or_p1_inv_r.restype = None
            lib.or_near_blocks.argtypes = [dp, i32p, ctypes.c_int, ctypes.c_int64, i64p, i64p, dp]
            lib.or_dl_kernel_matvec.argtypes = [ctypes.c_int64, dp, i64p, ctypes.c_int64, dp, dp,
                                                ctypes.c_double, ctypes.c_int64, dp, dp]
            lib.or_adl_kernel_matvec.argtypes = [ctypes.c_int64, dp, dp, i64p, ctypes.c_int64, dp,
                                                 ctypes.c_double, ctypes.c_int64, dp, dp]
            lib.or_p1_dn_inv_r.argtypes = [dp, dp, dp, dp, dp]
            lib.or_efie_near_blocks.argtypes = [dp, i32p, dp, ctypes.c_int, ctypes.c_int64, i64p, i64p, dp, dp]
            lib.or_p1_grad_inv_r.argtypes = [dp, dp, dp, dp, dp]
            lib.or_p1_grad_inv_r.restype = None
            lib.or_grad_cross_matvec.argtypes = [ctypes.c_int64, dp, i64p, ctypes.c_int64, dp, i64p, ctypes.c_double,
                                                 ctypes.c_int64, dp, dp]
            lib.or_mfie_near_blocks.argtypes = [dp, i32p, dp, ctypes.c_int, ctypes.c_int64, i64p, i64p, dp]
            lib.or_p1_dn_inv_r.restype = None
            lib.or_dl_near_blocks.argtypes = [dp, i32p, ctypes.c_int, ctypes.c_int64, i64p, i64p, dp]
            lib.or_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return int(_load().or_num_threads())


# --------------------------------------------------------------------------
# Sec. 3 / Sec. 4.2: quadrature and the P1 basis matrix
# --------------------------------------------------------------------------

def quad_rule(q: int):
    """Reference rule: barycentric points (q, 3) and weights (q,) summing to 1."""
    bary = np.zeros((q, 3))
    w = np.zeros(q)
    if _load().or_quad_rule(q, _dp(bary), _dp(w)) != 0:
        raise ValueError(f"no {q}-point rule (1, 3 or 7)")
    return bary, w


def triangle_areas(vtx, tri):
    a, b, c = vtx[tri[:, 0]], vtx[tri[:, 1]], vtx[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def quad_points(vtx, tri, q):
    """Quadrature points x_k (Nq, 3) and weights w_k (Nq,), k = t*q + j (Eq. approxA)."""
    bary, w = quad_rule(q)
    a, b, c = vtx[tri[:, 0]], vtx[tri[:, 1]], vtx[tri[:, 2]]
    x = (bary[None, :, 0:1] * a[:, None, :] + bary[None, :, 1:2] * b[:, None, :]
         + bary[None, :, 2:3] * c[:, None, :])
    wk = triangle_areas(vtx, tri)[:, None] * w[None, :]
    return x.reshape(-1, 3), wk.reshape(-1)


def basis_matrix(tri, nv, q):
    """Phi (Nq, Nv) with Phi_kj = phi_j(x_k): 3 nonzeros per row (Eq. WB)."""
    bary, _ = quad_rule(q)
    nt = tri.shape[0]
    rows = np.repeat(np.arange(nt * q), 3)
    cols = np.repeat(tri.astype(np.int64), q, axis=0).reshape(-1)
    vals = np.tile(bary.reshape(-1), nt)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nt * q, nv))


def mass_matrix(vtx, tri, q):
    """A = Phi^T W Phi (Eq. A=BWB)."""
    x, w = quad_points(vtx, tri, q)
    phi = basis_matrix(tri, vtx.shape[0], q)
    return (phi.T @ sp.diags(w) @ phi).tocsr()


# --------------------------------------------------------------------------
# Sec. 5: the dense kernel between point clouds
# --------------------------------------------------------------------------

def kernel_matvec(xt, tid, ys, u, k):
    """v = G u with G_tl = exp(ik r)/r, G = ik where tid[t] == l (u: (Ns, nrhs) complex)."""
    lib = _load()
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    u = np.asarray(u, dtype=np.complex128)
    if u.ndim == 1:
        u = u[:, None]
    nt, ns, nrhs = xt.shape[0], ys.shape[0], u.shape[1]
    uflat = np.ascontiguousarray(u.ravel(order="F"))     # column-major, interleaved re/im
    vflat = np.zeros(nt * nrhs, dtype=np.complex128)
    tidp = None
    if tid is not None:
        tid = np.ascontiguousarray(tid, dtype=np.int64)
        tidp = _i64p(tid)
    lib.or_kernel_matvec(nt, _dp(xt), tidp, ns, _dp(ys), float(k), nrhs,
                         _dp(uflat.view(np.float64)), _dp(vflat.view(np.float64)))
    return vflat.reshape((nt, nrhs), order="F")


def kernel_matrix(xt, tid, ys, k):
    """Dense G (Nt, Ns) complex."""
    lib = _load()
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    g = np.zeros((xt.shape[0], ys.shape[0]), dtype=np.complex128)
    tidp = None
    if tid is not None:
        tid = np.ascontiguousarray(tid, dtype=np.int64)
        tidp = _i64p(tid)
    lib.or_kernel_matrix(xt.shape[0], _dp(xt), tidp, ys.shape[0], _dp(ys), float(k), _dp(g.view(np.float64)))
    return g


# --------------------------------------------------------------------------
# Sec. 5.2: singular correction
# --------------------------------------------------------------------------

def p1_inv_r(x, p0, p1, p2):
    """int_T lambda_j(y)/|x-y| dy for j = 0, 1, 2 over T = (p0, p1, p2) (closed form)."""
    lib = _load()
    out = np.zeros(3)
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, p0, p1, p2)]
    lib.or_p1_inv_r(*[_dp(a) for a in args], _dp(out))
    return out


def near_pairs(tri, nv):
    """Ordered pairs (a, b) of triangles sharing at least one vertex, a == b included.

    Sorted by a, then b.
    """
    nt = tri.shape[0]
    inc = sp.csr_matrix((np.ones(3 * nt), (np.repeat(np.arange(nt), 3), tri.reshape(-1).astype(np.int64))),
                        shape=(nt, nv))
    adj = (inc @ inc.T).tocoo()
    order = np.lexsort((adj.col, adj.row))
    return adj.row[order].astype(np.int64), adj.col[order].astype(np.int64)


def near_blocks(vtx, tri, q, pa, pb):
    """3x3 correction block for each near pair (rows: test vertices of a, cols: trial of b)."""
    lib = _load()
    vtx = np.ascontiguousarray(vtx, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    out = np.zeros((pa.shape[0], 3, 3))
    if lib.or_near_blocks(_dp(vtx), _i32p(tri), int(q), pa.shape[0], _i64p(pa), _i64p(pb), _dp(out)) != 0:
        raise ValueError("bad quadrature order")
    return out


def near_matrix(vtx, tri, q):
    """Sparse real correction C (Nv, Nv): sum of the blocks placed at their vertex indices."""
    nv = vtx.shape[0]
    pa, pb = near_pairs(tri, nv)
    blk = near_blocks(vtx, tri, q, pa, pb)
    ti = tri[pa].astype(np.int64)  # (np, 3)
    tj = tri[pb].astype(np.int64)
    rows = np.repeat(ti, 3, axis=1).reshape(-1)
    cols = np.tile(tj, (1, 3)).reshape(-1)
    c = sp.coo_matrix((blk.reshape(-1), (rows, cols)), shape=(nv, nv)).tocsr()
    c.sum_duplicates()
    return c


# --------------------------------------------------------------------------
# Double layer: kernel n_y . grad_y exp(ikr)/r, correction 'grady[1/r]'
# --------------------------------------------------------------------------

def dl_kernel_matvec(xt, tid, ys, nrm, u, k):
    """v = H u with H_tl = (1 - ikr) exp(ikr) n_l . (x_t - y_l) / r^3, H = 0 where tid[t] == l."""
    lib = _load()
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    nrm = np.ascontiguousarray(nrm, dtype=np.float64)
    u = np.asarray(u, dtype=np.complex128)
    if u.ndim == 1:
        u = u[:, None]
    nt, ns, nrhs = xt.shape[0], ys.shape[0], u.shape[1]
    uflat = np.ascontiguousarray(u.ravel(order="F"))
    vflat = np.zeros(nt * nrhs, dtype=np.complex128)
    tidp = None
    if tid is not None:
        tid = np.ascontiguousarray(tid, dtype=np.int64)
        tidp = _i64p(tid)
    lib.or_dl_kernel_matvec(nt, _dp(xt), tidp, ns, _dp(ys), _dp(nrm), float(k), nrhs,
                            _dp(uflat.view(np.float64)), _dp(vflat.view(np.float64)))
    return vflat.reshape((nt, nrhs), order="F")


def adl_kernel_matvec(xt, nrm_t, tid, ys, u, k):
    """v = H' u with H'_tl = -(1 - ikr) exp(ikr) n_t . (x_t - y_l) / r^3 (normal at the
    target: n_x . grad_x exp(ikr)/r), H' = 0 where tid[t] == l."""
    lib = _load()
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    nrm_t = np.ascontiguousarray(nrm_t, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    u = np.asarray(u, dtype=np.complex128)
    if u.ndim == 1:
        u = u[:, None]
    nt, ns, nrhs = xt.shape[0], ys.shape[0], u.shape[1]
    uflat = np.ascontiguousarray(u.ravel(order="F"))
    vflat = np.zeros(nt * nrhs, dtype=np.complex128)
    tidp = None
    if tid is not None:
        tid = np.ascontiguousarray(tid, dtype=np.int64)
        tidp = _i64p(tid)
    lib.or_adl_kernel_matvec(nt, _dp(xt), _dp(nrm_t), tidp, ns, _dp(ys), float(k), nrhs,
                             _dp(uflat.view(np.float64)), _dp(vflat.view(np.float64)))
    return vflat.reshape((nt, nrhs), order="F")


def p1_grad_inv_r(x, p0, p1, p2):
    """int_T lambda_j(y) (x - y)/|x - y|^3 dy, (3, 3): row j, column the component (closed form)."""
    lib = _load()
    out = np.zeros(9)
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, p0, p1, p2)]
    lib.or_p1_grad_inv_r(*[_dp(a) for a in args], _dp(out))
    return out.reshape(3, 3)


def p1_dn_inv_r(x, p0, p1, p2):
    """int_T lambda_j(y) n . (x - y)/|x - y|^3 dy for j = 0, 1, 2 (closed form; 0 in the plane of T)."""
    lib = _load()
    out = np.zeros(3)
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, p0, p1, p2)]
    lib.or_p1_dn_inv_r(*[_dp(a) for a in args], _dp(out))
    return out


def dl_near_matrix(vtx, tri, q):
    """Sparse real double-layer correction (Nv, Nv) on the pairs sharing a vertex."""
    lib = _load()
    nv = vtx.shape[0]
    vtx = np.ascontiguousarray(vtx, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    pa, pb = near_pairs(tri, nv)
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    blk = np.zeros((pa.shape[0], 3, 3))
    if lib.or_dl_near_blocks(_dp(vtx), _i32p(tri), int(q), pa.shape[0], _i64p(pa), _i64p(pb), _dp(blk)) != 0:
        raise ValueError("bad quadrature order")
    ti, tj = tri[pa].astype(np.int64), tri[pb].astype(np.int64)
    rows = np.repeat(ti, 3, axis=1).reshape(-1)
    cols = np.tile(tj, (1, 3)).reshape(-1)
    c = sp.coo_matrix((blk.reshape(-1), (rows, cols)), shape=(nv, nv)).tocsr()
    c.sum_duplicates()
    return c


# --------------------------------------------------------------------------
# The operator on a mesh
# --------------------------------------------------------------------------

class Mesh:
    """Mesh + quadrature ``dom(mesh, q)`` and the P1 space on it (Sec. 4.1-4.3)."""

    def __init__(self, vtx, tri, q):
        self.vtx = np.ascontiguousarray(vtx, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.q = int(q)
        self.nv = self.vtx.shape[0]
        self.nt = self.tri.shape[0]
        self.x, self.w = quad_points(self.vtx, self.tri, self.q)
        self.nq = self.x.shape[0]
        self.phi = basis_matrix(self.tri, self.nv, self.q)
        self._c = None

    @property
    def near(self):
        if self._c is None:
            self._c = near_matrix(self.vtx, self.tri, self.q)
        return self._c

    def mass(self):
        return (self.phi.T @ sp.diags(self.w) @ self.phi).tocsr()

    def quad_ids_of_vertices(self, rows):
        """Quadrature points in the support of phi_i for each i in rows (sorted unique)."""
        sub = self.phi[:, np.asarray(rows)].tocsc()
        return np.unique(sub.indices)

    def far_apply(self, k, x, rows=None):
        """(1/4pi) Phi^T W_x G W_y Phi x, Eq. (BEM); rows: only these output rows (others 0)."""
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        u = self.w[:, None] * (self.phi @ x)                 # W_y Psi x
        if rows is None:
            tids = np.arange(self.nq)
        else:
            tids = self.quad_ids_of_vertices(rows)
        v = kernel_matvec(self.x[tids], tids, self.x, u, k)  # G (W_y Psi x), target rows tids
        vfull = np.zeros((self.nq, x.shape[1]), dtype=np.complex128)
        vfull[tids] = v
        y = (self.phi.T @ (self.w[:, None] * vfull)) / (4.0 * np.pi)  # Phi^T W_x (...)
        if rows is not None:
            mask = np.zeros(self.nv, dtype=bool)
            mask[np.asarray(rows)] = True
            y[~mask] = 0.0
        return y[:, 0] if one else y

    def point_normals(self):
        """Unit normal of the triangle of each quadrature point (Nq, 3)."""
        P = self.vtx[self.tri]
        n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        return np.repeat(n, self.q, axis=0)

    @property
    def dl_near(self):
        if getattr(self, "_cdl", None) is None:
            self._cdl = dl_near_matrix(self.vtx, self.tri, self.q)
        return self._cdl

    def dl_apply(self, k, x):
        """Galerkin double layer K x, K_ij = (1/4pi) int int phi_i(x) n_y . grad_y exp(ik|x-y|)/|x-y| phi_j(y):
        the same factorisation as the single layer (Phi^T W H W Phi / 4pi) with the
        kernel H and the 'grady[1/r]' correction on pairs sharing a vertex."""
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        u = self.w[:, None] * (self.phi @ x)
        v = dl_kernel_matvec(self.x, np.arange(self.nq), self.x, self.point_normals(), u, k)
        y = (self.phi.T @ (self.w[:, None] * v)) / (4.0 * np.pi) + self.dl_near @ x
        return y[:, 0] if one else y

    def adl_apply(self, k, x):
        """Galerkin adjoint double layer K' x, K'_ij = (1/4pi) int int phi_i(x) n_x . grad_x
        exp(ik|x-y|)/|x-y| phi_j(y): the kernel with the normal at the test point, and the
        transpose of the double layer's correction (K' = K^T for the Galerkin matrices, G
        being symmetric; the correction is taken as its discrete transpose)."""
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        u = self.w[:, None] * (self.phi @ x)
        v = adl_kernel_matvec(self.x, self.point_normals(), np.arange(self.nq), self.x, u, k)
        y = (self.phi.T @ (self.w[:, None] * v)) / (4.0 * np.pi) + self.dl_near.T @ x
        return y[:, 0] if one else y

    def cfie_apply(self, k, eta, x):
        """Direct combined-field operator (1/2 M + K' - i eta V) x for the sound-soft
        problem: its solution is the normal derivative of the total field, the density
        of the paper's first-kind system V lambda = F (Sec. 5.4)."""
        x = np.asarray(x, dtype=np.complex128)
        return 0.5 * (self.mass() @ x) + self.adl_apply(k, x) - 1j * eta * self.apply(k, x)

    def rhs_planewave_cfie(self, k, eta, dirs):
        """F_i = int phi_i (d/dn - i eta) exp(ik d.x) = int phi_i (ik d.n - i eta) exp(ik d.x)
        by the domain's rule, n the outward unit normal of each triangle."""
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        p = np.exp(1j * k * (self.x @ dirs.T)) * (1j * k * (self.point_normals() @ dirs.T) - 1j * eta)
        return np.asarray(self.phi.T @ (self.w[:, None] * p))

    def bw_apply(self, k, eta, x):
        """Brakhage-Werner combined operator (1/2 M + K - i eta V) x: the Galerkin
        exterior trace of u = (D - i eta S) phi (jump relation of the double-layer
        potential; Brakhage and Werner 1965), M = Phi^T W Phi (Eq. A=BWB)."""
        x = np.asarray(x, dtype=np.complex128)
        return 0.5 * (self.mass() @ x) + self.dl_apply(k, x) - 1j * eta * self.apply(k, x)

    def apply(self, k, x, rows=None):
        """V x = far part + C x (Sec. 5.2, listing of Sec. 5.4: LHS = integral + regularize)."""
        y = self.far_apply(k, x, rows)
        cx = self.near @ np.asarray(x, dtype=np.complex128)
        if rows is not None:
            mask = np.zeros(self.nv, dtype=bool)
            mask[np.asarray(rows)] = True
            cx[~mask] = 0.0
        return y + cx

    def assemble_far(self, k):
        g = kernel_matrix(self.x, np.arange(self.nq), self.x, k)
        pw = (sp.diags(self.w) @ self.phi).tocsr()           # W Phi
        return np.asarray((pw.T @ (pw.T @ g.T).T)) / (4.0 * np.pi)

    def assemble(self, k):
        """Dense V = (1/4pi) Phi^T W G W Phi + C (Nv, Nv) complex."""
        return self.assemble_far(k) + self.near.toarray()

    def potential(self, k, pts, x):
        """Single-layer potential of the density x (nv, nrhs) at points pts (npts, 3):
        the radiation operator of the listing in Sec. 5.4,
        integral(points, S2, Gxy, Vh)/(4 pi) + regularize(points, S2, '[1/r]', Vh)/(4 pi).
        The Gauss-point sum of exp(ikr)/r; then, for each triangle whose centroid
        lies within twice its largest centroid-vertex distance of the point (the
        reading of "close enough" for points), the closed-form integral of
        lambda_j / |x - y| over it minus the Gauss sum of the same (Sec. 5.2).
        Points must not coincide with Gauss points."""
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
        u = self.w[:, None] * (self.phi @ x)
        v = kernel_matvec(pts, None, self.x, u, k)
        bary, _ = quad_rule(self.q)
        P = self.vtx[self.tri]                                  # (nt, 3, 3)
        cen = P.mean(axis=1)
        rad2 = 4.0 * np.max(np.sum((P - cen[:, None, :]) ** 2, axis=2), axis=1)
        for i, p in enumerate(pts):
            for b in np.flatnonzero(np.sum((cen - p) ** 2, axis=1) < rad2):
                exact = p1_inv_r(p, *P[b])
                ys = self.x[b * self.q:(b + 1) * self.q]
                r = np.linalg.norm(ys - p, axis=1)
                keep = r > 0.0
                gauss = (self.w[b * self.q:(b + 1) * self.q][keep] / r[keep]) @ bary[keep]
                v[i] += (exact - gauss) @ x[self.tri[b]]
        v /= 4.0 * np.pi
        return v[:, 0] if one else v

    def rhs_planewave(self, k, dirs):
        """F_i = int phi_i exp(ik d.x) by the domain's rule, one column per direction (Sec. 5.4)."""
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        p = np.exp(1j * k * (self.x @ dirs.T))               # (Nq, nd)
        return np.asarray(self.phi.T @ (self.w[:, None] * p))


# --------------------------------------------------------------------------
# EFIE with RWG functions (the electromagnetic listing of Sec. 5.5):
#   T = ik/(4pi) int int phi_m . phi_n G - i/(4pi k) int int div phi_m div phi_n G
#     + the same two terms with the '[1/r]' regularisation (Sec. 5.2)
# --------------------------------------------------------------------------

def rwg_topology(tri, nv):
    """RWG functions of a closed, consistently oriented mesh, one per edge.

    Edges are the vertex pairs (a < b) in lexicographic order.  In triangle
    t = (v0, v1, v2) the local edge j runs v_{j+1} -> v_{j+2}, opposite v_j; t is
    the edge's plus triangle (sign +1) where the edge runs a -> b, its minus
    triangle (sign -1) where it runs b -> a.  Returns edges (nE, 2), tedge (nt, 3)
    edge ids and tsign (nt, 3)."""
    tri = np.asarray(tri, dtype=np.int64)
    a, b = tri[:, [1, 2, 0]], tri[:, [2, 0, 1]]
    key = np.minimum(a, b) * nv + np.maximum(a, b)
    uniq, inv, counts = np.unique(key.reshape(-1), return_inverse=True, return_counts=True)
    if np.any(counts != 2):
        raise ValueError("RWG functions need a closed mesh (every edge in two triangles)")
    tsign = np.where(a < b, 1.0, -1.0)
    plus = np.zeros(uniq.shape[0])
    np.add.at(plus, inv, tsign.reshape(-1))
    if np.any(plus != 0.0):
        raise ValueError("inconsistent orientation: an edge runs the same way in both triangles")
    edges = np.stack([uniq // nv, uniq % nv], axis=1)
    return edges, inv.reshape(tri.shape), tsign


def rwg_eval(P, j, s, y):
    """The RWG function of local edge j of the triangle P (3 x 3) with sign s at the
    points y (n, 3): s l_j / (2 A) (y - P_j), and its divergence s l_j / A."""
    A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    l = np.linalg.norm(P[(j + 2) % 3] - P[(j + 1) % 3])
    return s * l / (2.0 * A) * (np.atleast_2d(y) - P[j]), s * l / A


def rwg_basis(vtx, tri, q):
    """Phi_c (Nq, nE), c = 0, 1, 2: the vector components of the RWG functions at
    the Gauss points, and Dv (Nq, nE) their divergence; 3 nonzeros per row."""
    vtx = np.asarray(vtx, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    nt = tri.shape[0]
    edges, tedge, tsign = rwg_topology(tri, vtx.shape[0])
    x, _ = quad_points(vtx, tri, q)
    rows, cols, vals, dvals = [], [], [[], [], []], []
    for t in range(nt):
        P = vtx[tri[t]]
        pts = x[t * q:(t + 1) * q]
        for j in range(3):
            f, d = rwg_eval(P, j, tsign[t, j], pts)
            rows.append(np.arange(t * q, (t + 1) * q))
            cols.append(np.full(q, tedge[t, j]))
            for c in range(3):
                vals[c].append(f[:, c])
            dvals.append(np.full(q, d))
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    ne = edges.shape[0]
    phi = [sp.csr_matrix((np.concatenate(vals[c]), (rows, cols)), shape=(nt * q, ne)) for c in range(3)]
    dv = sp.csr_matrix((np.concatenate(dvals), (rows, cols)), shape=(nt * q, ne))
    return phi, dv


def efie_near_matrices(vtx, tri, q):
    """CA, CB (nE, nE) real: on every ordered pair (a, b) of triangles sharing a
    vertex, for each Gauss point x_k of a, the analytic int_b f / |x_k - y| minus the
    Gauss sum over b's points (the point itself left out), paired with w_k times the
    test function of a:  CA with f = phi_j^b (dotted with phi_i^a(x_k)), CB with
    f = div phi_j^b (times div phi_i^a).  The analytic integrals follow from the P1
    ones: phi_j = s l_j / (2A) sum_m lambda_m (P_m - P_j) on b (C, or_efie_near_blocks)."""
    lib = _load()
    vtx = np.ascontiguousarray(vtx, dtype=np.float64)
    tri32 = np.ascontiguousarray(tri, dtype=np.int32)
    nv = vtx.shape[0]
    edges, tedge, tsign = rwg_topology(tri32, nv)
    tsign = np.ascontiguousarray(tsign, dtype=np.float64)
    pa, pb = near_pairs(tri32, nv)
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    ba = np.zeros((pa.shape[0], 3, 3))
    bb = np.zeros((pa.shape[0], 3, 3))
    if lib.or_efie_near_blocks(_dp(vtx), _i32p(tri32), _dp(tsign), int(q), pa.shape[0], _i64p(pa), _i64p(pb),
                               _dp(ba), _dp(bb)) != 0:
        raise ValueError("bad quadrature order")
    rows = np.repeat(tedge[pa], 3, axis=1).reshape(-1)
    cols = np.tile(tedge[pb], (1, 3)).reshape(-1)
    ne = edges.shape[0]
    CA = sp.coo_matrix((ba.reshape(-1), (rows, cols)), shape=(ne, ne)).tocsr()
    CB = sp.coo_matrix((bb.reshape(-1), (rows, cols)), shape=(ne, ne)).tocsr()
    CA.sum_duplicates()
    CB.sum_duplicates()
    return CA, CB


def efie_near_matrices_py(vtx, tri, q):
    """The same matrices from a direct loop over pairs and Gauss points in numpy
    (slow; a cross-check of the C form on small meshes)."""
    vtx = np.asarray(vtx, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    nv = vtx.shape[0]
    edges, tedge, tsign = rwg_topology(tri, nv)
    x, w = quad_points(vtx, tri, q)
    pa, pb = near_pairs(tri, nv)
    ne = edges.shape[0]
    ra, rb, va, vb = [], [], [], []
    for a, b in zip(pa, pb):
        Pa, Pb = vtx[tri[a]], vtx[tri[b]]
        xa, wa = x[a * q:(a + 1) * q], w[a * q:(a + 1) * q]
        yb, wb = x[b * q:(b + 1) * q], w[b * q:(b + 1) * q]
        Ab = 0.5 * np.linalg.norm(np.cross(Pb[1] - Pb[0], Pb[2] - Pb[0]))
        for kk in range(q):
            I = p1_inv_r(xa[kk], Pb[0], Pb[1], Pb[2])          # int_b lambda_m / R
            r = np.linalg.norm(yb - xa[kk], axis=1)
            inv = np.zeros(q)
            mask = r > 0.0
            if a == b:
                mask[kk] = False                                  # the point itself
            inv[mask] = wb[mask] / r[mask]
            for jb in range(3):
                sj = tsign[b, jb]
                lj = np.linalg.norm(Pb[(jb + 2) % 3] - Pb[(jb + 1) % 3])
                vec_an = sj * lj / (2.0 * Ab) * (I[:, None] * (Pb - Pb[jb])).sum(axis=0)
                div_an = sj * lj / Ab * I.sum()
                fb, db = rwg_eval(Pb, jb, sj, yb)
                vec_g = (inv[:, None] * fb).sum(axis=0)
                div_g = db * inv.sum()
                for ia in range(3):
                    fa, da = rwg_eval(Pa, ia, tsign[a, ia], xa[kk])
                    ra.append(tedge[a, ia])
                    rb.append(tedge[b, jb])
                    va.append(wa[kk] * float(fa[0] @ (vec_an - vec_g)))
                    vb.append(wa[kk] * da * (div_an - div_g))
    CA = sp.coo_matrix((va, (ra, rb)), shape=(ne, ne)).tocsr()
    CB = sp.coo_matrix((vb, (ra, rb)), shape=(ne, ne)).tocsr()
    CA.sum_duplicates()
    CB.sum_duplicates()
    return CA, CB


def grad_cross_matvec(xt, tri_t, ys, tri_s, u, k):
    """v_t = sum_l F(r_tl) (x_t - y_l) x u_l, F = (1 - ikr) exp(ikr)/r^3 (grad_y exp(ikr)/r =
    F (x - y)), pairs with tri_t[t] == tri_s[l] left out; u: (ns, 3, nrhs) complex -> (nt, 3, nrhs)."""
    lib = _load()
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    tri_t = np.ascontiguousarray(tri_t, dtype=np.int64)
    tri_s = np.ascontiguousarray(tri_s, dtype=np.int64)
    u = np.asarray(u, dtype=np.complex128)
    nt, ns, nrhs = xt.shape[0], ys.shape[0], u.shape[2]
    uflat = np.ascontiguousarray(np.transpose(u, (2, 1, 0)).reshape(-1))   # ((3 j + c) ns + l)
    vflat = np.zeros(nt * 3 * nrhs, dtype=np.complex128)
    lib.or_grad_cross_matvec(nt, _dp(xt), _i64p(tri_t), ns, _dp(ys), _i64p(tri_s), float(k), nrhs,
                             _dp(uflat.view(np.float64)), _dp(vflat.view(np.float64)))
    return np.transpose(vflat.reshape(nrhs, 3, nt), (2, 1, 0))


def mfie_near_matrix(vtx, tri, q):
    """C (nE, nE) real, the MFIE's 'grady[1/r]' correction (times 1/(4pi)) on every ordered
    pair of triangles sharing a vertex (0 inside one triangle; C, or_mfie_near_blocks)."""
    lib = _load()
    vtx = np.ascontiguousarray(vtx, dtype=np.float64)
    tri32 = np.ascontiguousarray(tri, dtype=np.int32)
    nv = vtx.shape[0]
    edges, tedge, tsign = rwg_topology(tri32, nv)
    tsign = np.ascontiguousarray(tsign, dtype=np.float64)
    pa, pb = near_pairs(tri32, nv)
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    blk = np.zeros((pa.shape[0], 3, 3))
    if lib.or_mfie_near_blocks(_dp(vtx), _i32p(tri32), _dp(tsign), int(q), pa.shape[0], _i64p(pa), _i64p(pb),
                               _dp(blk)) != 0:
        raise ValueError("bad quadrature order")
    rows = np.repeat(tedge[pa], 3, axis=1).reshape(-1)
    cols = np.tile(tedge[pb], (1, 3)).reshape(-1)
    ne = edges.shape[0]
    c = sp.coo_matrix((blk.reshape(-1), (rows, cols)), shape=(ne, ne)).tocsr()
    c.sum_duplicates()
    return c


class EfieMesh(Mesh):
    """The mesh with the RWG space ``fem(mesh, 'RWG')`` on ``dom(mesh, q)``."""

    def __init__(self, vtx, tri, q):
        super().__init__(vtx, tri, q)
        self.edges, self.tedge, self.tsign = rwg_topology(self.tri, self.nv)
        self.ne = self.edges.shape[0]
        self.rwg, self.div = rwg_basis(self.vtx, self.tri, self.q)
        self._cab = None

    @property
    def efie_near(self):
        if self._cab is None:
            self._cab = efie_near_matrices(self.vtx, self.tri, self.q)
        return self._cab

    def efie_apply(self, k, x):
        """T x, T = ik/(4pi) sum_c Phi_c^T W G W Phi_c - i/(4pi k) Dv^T W G W Dv
        + ik/(4pi) CA - i/(4pi k) CB (the listing's T with its two regularize terms);
        x: (nE,) or (nE, nrhs) complex; k > 0."""
        if not k > 0.0:
            raise ValueError("the EFIE needs k > 0")
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        nrhs = x.shape[1]
        u = np.concatenate([self.w[:, None] * (f @ x) for f in (*self.rwg, self.div)], axis=1)
        v = kernel_matvec(self.x, np.arange(self.nq), self.x, u, k)
        wv = self.w[:, None] * v
        vec = sum(self.rwg[c].T @ wv[:, c * nrhs:(c + 1) * nrhs] for c in range(3))
        dv = self.div.T @ wv[:, 3 * nrhs:]
        CA, CB = self.efie_near
        y = 1j * k / (4.0 * np.pi) * (vec + CA @ x) - 1j / (4.0 * np.pi * k) * (dv + CB @ x)
        return y[:, 0] if one else y

    @property
    def mfie_near(self):
        if getattr(self, "_cm", None) is None:
            self._cm = mfie_near_matrix(self.vtx, self.tri, self.q)
        return self._cm

    def rwg_mass(self):
        """Id = int phi_m . phi_n by the domain's rule (the listing's integral(sigma, Vh, Vh))."""
        return sum(self.rwg[c].T @ sp.diags(self.w) @ self.rwg[c] for c in range(3)).tocsr()

    def mfie_apply(self, k, x):
        """nxK x = (1/4pi) sum_k w_k (n_k x phi_m(x_k)) . sum_l F (x_k - y_l) x (w_l J(y_l)) + C x,
        J = sum_n x_n phi_n, F (x - y) = grad_y exp(ik|x-y|)/|x-y| (the listing's nxK)."""
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        u = np.stack([self.w[:, None] * (self.rwg[c] @ x) for c in range(3)], axis=1)   # (nq, 3, nrhs)
        tid = np.repeat(np.arange(self.nt), self.q)
        v = grad_cross_matvec(self.x, tid, self.x, tid, u, k)
        n = self.point_normals()
        vxn = np.cross(v, n[:, :, None], axis=1)             # (n x phi) . v = phi . (v x n)
        y = sum(self.rwg[c].T @ (self.w[:, None] * vxn[:, c, :]) for c in range(3)) / (4.0 * np.pi)
        y = y + self.mfie_near @ x
        return y[:, 0] if one else y

    def emcfie_apply(self, k, beta, x):
        """The listing's LHS: -beta T + (1 - beta) (1/2 Id - nxK)."""
        x = np.asarray(x, dtype=np.complex128)
        out = (1.0 - beta) * (0.5 * (self.rwg_mass() @ x) - self.mfie_apply(k, x))
        if beta != 0.0:
            out = out - beta * self.efie_apply(k, x)
        return out

    def rhs_planewave_mfie(self, k, dirs, pols):
        """int (n x phi_m) . H_inc = int phi_m . (H_inc x n), H_inc = (d x p) exp(ik d.x)."""
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        pols = np.atleast_2d(np.asarray(pols, dtype=np.float64))
        hp = np.cross(dirs, pols)                             # (nd, 3)
        e = np.exp(1j * k * (self.x @ dirs.T))                # (nq, nd)
        hxn = np.cross(hp[None, :, :], self.point_normals()[:, None, :])   # (nq, nd, 3)
        return np.asarray(sum(self.rwg[c].T @ (self.w[:, None] * e * hxn[:, :, c]) for c in range(3)))

    def rhs_planewave_emcfie(self, k, beta, dirs, pols):
        """The listing's RHS: beta int phi . E_inc - (1 - beta) int (n x phi) . H_inc."""
        return beta * self.rhs_planewave_efie(k, dirs, pols) - (1.0 - beta) * self.rhs_planewave_mfie(k, dirs, pols)

    def rhs_planewave_efie(self, k, dirs, pols):
        """F_m = int phi_m . p exp(ik d.x) by the domain's rule, one column per
        (direction d_j, polarisation p_j) (the listing's integral(sigma, Vh, PWE))."""
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        pols = np.atleast_2d(np.asarray(pols, dtype=np.float64))
        e = np.exp(1j * k * (self.x @ dirs.T))                   # (Nq, nd)
        comp = sum(self.rwg[c].T @ (self.w[:, None] * e * pols[None, :, c]) for c in range(3))
        return np.asarray(comp)


def mie_pec_amplitudes(k, cos_theta):
    """S1, S2 of a perfectly conducting unit sphere (Mie series in the
    perfectly-conducting limit: a_n = psi_n'(k)/xi_n'(k), b_n = psi_n(k)/xi_n(k),
    psi_n(x) = x j_n(x), xi_n(x) = x h_n(x)); the angle functions pi_n, tau_n by
    their recurrences."""
    from scipy.special import spherical_jn, spherical_yn
    mu = np.asarray(cos_theta, dtype=np.float64)
    nmax = int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 10))
    s1 = np.zeros(mu.shape, dtype=np.complex128)
    s2 = np.zeros(mu.shape, dtype=np.complex128)
    pi_prev, pi_cur = np.zeros_like(mu), np.ones_like(mu)   # pi_0, pi_1
    for n in range(1, nmax + 1):
        if n > 1:
            pi_prev, pi_cur = pi_cur, ((2 * n - 1) * mu * pi_cur - n * pi_prev) / (n - 1)
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        j, jp = spherical_jn(n, k), spherical_jn(n, k, derivative=True)
        h = j + 1j * spherical_yn(n, k)
        hp = jp + 1j * spherical_yn(n, k, derivative=True)
        psi, dpsi = k * j, j + k * jp
        xi, dxi = k * h, h + k * hp
        an, bn = dpsi / dxi, psi / xi
        c = (2 * n + 1) / (n * (n + 1))
        s1 += c * (an * pi_cur + bn * tau)
        s2 += c * (an * tau + bn * pi_cur)
    return s1, s2


# --------------------------------------------------------------------------
# Solvers
# --------------------------------------------------------------------------

def solve_lu(a, f):
    """Direct solve (the paper's LHS \\ RHS, Sec. 5.4)."""
    return np.linalg.solve(a, f)


def gmres(matvec, f, tol=1e-6, restart=200, maxit=2000, x0=None):
    """Restarted GMRES for one right-hand side: Arnoldi with classical Gram-Schmidt
    applied twice, Givens rotations, stop when ||f - A x|| <= tol ||f||.

    Returns (x, iterations, true relative residual).
    """
    f = np.asarray(f, dtype=np.complex128)
    n = f.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxit:
        r = f - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * fn:
            break
        m = min(restart, maxit - it)
        Q = np.zeros((n, m + 1), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Q[:, 0] = r / beta
        j_end = 0
        for j in range(m):
            w = matvec(Q[:, j])
            h = Q[:, : j + 1].conj().T @ w
            w = w - Q[:, : j + 1] @ h
            h2 = Q[:, : j + 1].conj().T @ w
            w = w - Q[:, : j + 1] @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                Q[:, j + 1] = w / hn
            # unitary rotations [[conj(c), conj(s)], [-s, c]] with c = a/den, s = b/den
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, b = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = a / den
                sn[j] = b / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_end = j + 1
            if abs(g[j + 1]) <= tol * fn or hn == 0:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + Q[:, :j_end] @ y
    res = np.linalg.norm(f - matvec(x)) / fn
    return x, it, res


# --------------------------------------------------------------------------
# Closed forms on the unit sphere
# --------------------------------------------------------------------------

def sphere_eigenvalue(n: int, k: float) -> complex:
    """Single-layer eigenvalue on the unit sphere for degree-n harmonics:
    1/(2n+1) at k = 0, else i k j_n(k) h_n^(1)(k)."""
    from scipy.special import spherical_jn, spherical_yn
    if k == 0.0:
        return 1.0 / (2 * n + 1)
    j = spherical_jn(n, k)
    return 1j * k * j * (j + 1j * spherical_yn(n, k))


def mie_density(k: float, d, pts):
    """Density lambda of V lambda = F on the unit sphere for p_inc = exp(ik d.x):
    lambda(x) = sum_n (2n+1) i^n P_n(d.x) / (i k h_n^(1)(k))."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    pts = np.asarray(pts, dtype=np.float64)
    c = (pts / np.linalg.norm(pts, axis=1, keepdims=True)) @ d
    nmax = int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 10))
    lam = np.zeros(pts.shape[0], dtype=np.complex128)
    for n in range(nmax + 1):
        h = spherical_jn(n, k) + 1j * spherical_yn(n, k)
        lam += (2 * n + 1) * (1j ** n) * eval_legendre(n, c) / (1j * k * h)
    return lam


def dl_sphere_eigenvalue(n: int, k: float) -> complex:
    """Double-layer eigenvalue on the unit sphere for degree-n harmonics (outward
    normal): -1/(2(2n+1)) at k = 0, else 1/2 + i k^2 j_n(k) h_n^(1)'(k)."""
    from scipy.special import spherical_jn, spherical_yn
    if k == 0.0:
        return -1.0 / (2 * (2 * n + 1))
    hp = spherical_jn(n, k, derivative=True) + 1j * spherical_yn(n, k, derivative=True)
    return 0.5 + 1j * k * k * spherical_jn(n, k) * hp


def bw_density(k: float, eta: float, d, pts):
    """Density phi of (1/2 + K - i eta V) phi = -p_inc on the unit sphere for
    p_inc = exp(ik d.x) = sum_n (2n+1) i^n j_n(k) P_n(d.x):
    phi(x) = -sum_n (2n+1) i^n j_n(k) P_n(d.x) / (1/2 + mu_n(K) - i eta mu_n(V))."""
    from scipy.special import eval_legendre, spherical_jn
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    pts = np.asarray(pts, dtype=np.float64)
    c = (pts / np.linalg.norm(pts, axis=1, keepdims=True)) @ d
    nmax = int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 10))
    phi = np.zeros(pts.shape[0], dtype=np.complex128)
    for n in range(nmax + 1):
        lam = 0.5 + dl_sphere_eigenvalue(n, k) - 1j * eta * sphere_eigenvalue(n, k)
        phi -= (2 * n + 1) * (1j ** n) * spherical_jn(n, k) * eval_legendre(n, c) / lam
    return phi
