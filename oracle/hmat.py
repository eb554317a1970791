"""Compressed far field of the single layer, plain FP64 (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path.

Sec. 5.3 of the paper couples the BEM matrices with a hierarchical
(H-matrix) compression to a tolerance ``tol``: far-apart groups of unknowns
interact through low-rank blocks, built from a few rows and columns of the
block.  This module computes that idea on one level of a cluster tree (a
block low-rank matrix), step by step:

1. Clusters: recursive coordinate bisection of the vertices (split the
   bounding box of the vertices along its longest side at the median) until a
   cluster holds at most ``leaf`` vertices.
2. Each cluster's box covers the supports of its basis functions: every vertex
   of every triangle that touches one of its vertices.
3. A pair of clusters (s, t) is admissible when
   dist(box_s, box_t) >= eta * max(diam_s, diam_t).
4. The block of V_far = (1/4pi) Phi^T W G W Phi for an admissible pair is
   replaced by the adaptive cross approximation with partial pivoting
   (Bebendorf 2000): U W^T from rows and columns of the block, stopped when the
   newest rank-one term is below eps times the Frobenius norm of the sum;
   the other blocks stay dense.
5. Apply: y_s = sum_t B_st x_t.

The block entries come from the same Gauss-point kernel as the oracle's
dense far part (Sec. 5, Eq. (BEM)); the singular correction C is not part of
the compressed operator and is added by the caller.
"""
from __future__ import annotations

import numpy as np

from . import kernel_matrix


def bisect_clusters(vtx, leaf):
    """Leaf clusters (index arrays) of a recursive coordinate bisection."""
    out = []

    def rec(idx):
        if len(idx) <= leaf:
            out.append(np.sort(idx))
            return
        p = vtx[idx]
        axis = int(np.argmax(p.max(axis=0) - p.min(axis=0)))
        order = idx[np.argsort(p[:, axis], kind="stable")]
        h = len(order) // 2
        rec(order[:h])
        rec(order[h:])

    rec(np.arange(vtx.shape[0]))
    return out


def support_boxes(vtx, tri, clusters):
    """Bounding box (lo, hi) of the supports of each cluster's basis functions."""
    nv = vtx.shape[0]
    owner = np.empty(nv, dtype=np.int64)
    for c, idx in enumerate(clusters):
        owner[idx] = c
    lo = np.full((len(clusters), 3), np.inf)
    hi = np.full((len(clusters), 3), -np.inf)
    for t in tri:
        p = vtx[t]
        for c in set(owner[t].tolist()):
            lo[c] = np.minimum(lo[c], p.min(axis=0))
            hi[c] = np.maximum(hi[c], p.max(axis=0))
    return lo, hi


def admissible(lo, hi, s, t, eta):
    gap = np.maximum(0.0, np.maximum(lo[s] - hi[t], lo[t] - hi[s]))
    dist = np.linalg.norm(gap)
    diam = max(np.linalg.norm(hi[s] - lo[s]), np.linalg.norm(hi[t] - lo[t]))
    return dist >= eta * diam


def aca(A, eps, rmax=None):
    """Adaptive cross approximation with partial pivoting of a complex block:
    A ~ U @ W.T, U (m, r), W (n, r).  Rows are taken as pivots in turn (the
    largest entry of the newest column among the rows not used yet); the
    Frobenius norm of the approximation is updated exactly from the inner
    products of the terms; stops when |u_r| |w_r| <= eps |U W^T|_F."""
    m, n = A.shape
    rmax = min(m, n) if rmax is None else rmax
    U = np.zeros((m, 0), dtype=np.complex128)
    W = np.zeros((n, 0), dtype=np.complex128)
    used_r = np.zeros(m, dtype=bool)
    used_c = np.zeros(n, dtype=bool)
    s2 = 0.0
    i = 0
    while U.shape[1] < rmax:
        row = A[i, :] - U[i, :] @ W.T
        used_r[i] = True
        mag = np.abs(row)
        mag[used_c] = -1.0
        j = int(np.argmax(mag))
        if mag[j] <= 0.0:
            free = np.flatnonzero(~used_r)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        w = row / row[j]
        u = A[:, j] - U @ W[j, :]
        used_c[j] = True
        cross = (U.conj().T @ u) * (W.conj().T @ w)
        s2 += float(np.vdot(u, u).real * np.vdot(w, w).real + 2.0 * np.sum(cross).real)
        U = np.column_stack([U, u])
        W = np.column_stack([W, w])
        if np.linalg.norm(u) * np.linalg.norm(w) <= eps * np.sqrt(max(s2, 0.0)):
            break
        mag = np.abs(u)
        mag[used_r] = -1.0
        i = int(np.argmax(mag))
        if mag[i] < 0.0:
            break
    return U, W


class CompressedFar:
    """Block low-rank V_far of an oracle Mesh at wavenumber k (FP64)."""

    def __init__(self, mesh, k, eps=1e-5, leaf=64, eta=1.0, vfar=None):
        """vfar: the dense far part (mesh.assemble_far(k)) to slice blocks from
        (small meshes); without it each block is computed from its points."""
        self.mesh, self.k, self.eps = mesh, float(k), float(eps)
        self.clusters = bisect_clusters(mesh.vtx, leaf)
        lo, hi = support_boxes(mesh.vtx, mesh.tri, self.clusters)
        pw = (mesh.phi.T.multiply(mesh.w[None, :])).tocsr()  # (W Phi)^T: (nv, nq)
        self._pw = pw
        self.blocks = []  # (s, t, kind, data)
        nc = len(self.clusters)
        for s in range(nc):
            for t in range(nc):
                if vfar is not None:
                    blk = vfar[np.ix_(self.clusters[s], self.clusters[t])]
                else:
                    blk = self.block(s, t)
                if s != t and admissible(lo, hi, s, t, eta):
                    U, W = aca(blk, self.eps)
                    self.blocks.append((s, t, "lowrank", (U, W)))
                else:
                    self.blocks.append((s, t, "dense", blk))

    def points_of(self, s):
        """Quadrature points in the support of cluster s's basis functions."""
        sub = self._pw[self.clusters[s], :]
        return np.unique(sub.indices)

    def block(self, s, t):
        """Exact block V_far[cluster s, cluster t]."""
        ps, pt = self.points_of(s), self.points_of(t)
        pos = {int(p): n for n, p in enumerate(pt)}
        tid = np.array([pos.get(int(p), -1) for p in ps], dtype=np.int64)
        g = kernel_matrix(self.mesh.x[ps], tid, self.mesh.x[pt], self.k)
        a = self._pw[self.clusters[s], :][:, ps].toarray()
        b = self._pw[self.clusters[t], :][:, pt].toarray()
        return a @ g @ b.T / (4.0 * np.pi)

    def ranks(self):
        return [d[0].shape[1] for _, _, kind, d in self.blocks if kind == "lowrank"]

    def stored_entries(self):
        n = 0
        for _, _, kind, d in self.blocks:
            n += d.size if kind == "dense" else d[0].size + d[1].size
        return n

    def apply(self, x):
        x = np.asarray(x, dtype=np.complex128)
        one = x.ndim == 1
        if one:
            x = x[:, None]
        y = np.zeros((self.mesh.nv, x.shape[1]), dtype=np.complex128)
        for s, t, kind, d in self.blocks:
            xs = x[self.clusters[t]]
            if kind == "dense":
                y[self.clusters[s]] += d @ xs
            else:
                U, W = d
                y[self.clusters[s]] += U @ (W.T @ xs)
        return y[:, 0] if one else y
