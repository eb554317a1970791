"""Training and evaluation of the learned preconditioner (control flow only).

Every numerical step runs in libgyps: the correction pairs come from the
library's own GMRES solves, the gradients and Adam steps from
gyps_precond_train_step, the evaluation from gyps_gmres_solve with and without
the network.  The random residuals are drawn on the host from seeded
generators and passed in.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

import paper_1804_00995_gb300 as g
import synth


@dataclass
class Pair:
    mesh: "g.Mesh"
    k: float
    R: object  # (nv, B) complex128 device tensor
    E: object  # V^{-1} R to the generation tolerance


@dataclass
class TrainLog:
    losses: list = field(default_factory=list)
    seconds: float = 0.0
    steps: int = 0


def random_meshes(seed: int, count: int, levels=(4, 5), k_range=(4.0, 16.0), q: int = 3):
    """Random-axis ellipsoids (semi-axes U[0.5, 2]) at the given icosphere levels, k ~ U[k_range]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        lv = int(rng.choice(levels))
        v, t, ax = synth.random_ellipsoid(rng, lv)
        k = float(rng.uniform(*k_range))
        out.append((g.Mesh(v, t, q), k, dict(level=lv, axes=ax.tolist(), vtx=v, tri=t)))
    return out


def make_pairs(meshes, nrhs: int = 16, tol: float = 1e-2, maxit: int = 400, seed: int = 0, redraw: int = 2,
               k_range=(4.0, 16.0)):
    """For each mesh, nrhs residual-like right-hand sides (complex white noise)
    and their solutions of V E = R by the library's GMRES (working precision
    FP32 or tensor cores, FP32 check).  Only columns whose solve reached tol
    are kept (near an interior resonance of the surface GMRES stalls and the
    'correction' would be noise); a mesh with no converged column is solved
    again at a new k ~ U[k_range] (at most `redraw` times).
    Returns (pairs, stats) with stats per mesh: iterations, kept columns, k."""
    import torch
    rng = np.random.default_rng(seed)
    pairs, stats = [], []
    for mesh, k, _ in meshes:
        for attempt in range(redraw + 1):
            R = torch.as_tensor(synth.random_complex(rng, mesh.nv, nrhs)).to(mesh.device).t().contiguous().t()
            E, rep = g.gmres_solve(mesh, k, R, tol=tol, restart=100, maxit=maxit, prec="auto", check_prec="fp32",
                                   max_refine=0)
            keep = np.flatnonzero(rep.converged)
            if keep.size or attempt == redraw:
                break
            k = float(rng.uniform(*k_range))
        stats.append(dict(iterations=rep.iterations, kept=int(keep.size), k=k))
        if keep.size:
            idx = torch.as_tensor(keep, device=R.device)
            pairs.append(Pair(mesh, k, R[:, idx].t().contiguous().t(), E[:, idx].t().contiguous().t()))
    return pairs, stats


def make_krylov_pairs(meshes, ndirs: int = 4, steps=(5, 15, 40), tol: float = 1e-5, maxit: int = 600, seed: int = 0):
    """Pairs from the solver's own Krylov iterations.  For plane-wave
    right-hand sides F (ndirs random directions) on each mesh: the GMRES
    solution X* (to tol) and the iterates X_m after m GMRES steps from zero
    (m in `steps`).  The errors E_m = X* - X_m and their residuals
    R_m = V E_m (one apply, so each pair is exact whatever tol) are the inputs
    and corrections that flexible GMRES hands the network.  Columns whose
    solve stalls (near an interior resonance) give no pairs.
    Returns (pairs, stats) like make_pairs."""
    import torch
    rng = np.random.default_rng(seed)
    pairs, stats = [], []
    for mesh, k, _ in meshes:
        F = g.rhs_planewave(mesh, k, synth.plane_wave_dirs(rng, ndirs))
        Xs, rep = g.gmres_solve(mesh, k, F, tol=tol, restart=100, maxit=maxit, prec="auto", check_prec="fp32",
                                max_refine=0)
        keep = np.flatnonzero(rep.converged)
        stats.append(dict(iterations=rep.iterations, kept=int(keep.size) * len(steps), k=k))
        if not keep.size:
            continue
        idx = torch.as_tensor(keep, device=Xs.device)
        Rs, Es = [], []
        for m in steps:
            Xm, _ = g.gmres_solve(mesh, k, F, tol=1e-14, restart=m, maxit=m, prec="auto", check_prec="fp32",
                                  max_refine=0)
            E = (Xs[:, idx] - Xm[:, idx]).t().contiguous().t()
            Rs.append(g.sl_apply(mesh, k, E, prec="fp32"))
            Es.append(E)
        R = torch.cat(Rs, dim=1).t().contiguous().t()
        E = torch.cat(Es, dim=1).t().contiguous().t()
        pairs.append(Pair(mesh, k, R, E))
    return pairs, stats


def train(P: "g.Precond", pairs, steps: int, lr: float = 1e-3, batch: int = 16, seed: int = 0, log_every: int = 50,
          lr_final: float = 1e-4):
    """Adam on random minibatches (columns of one pair set), cosine-free
    geometric decay from lr to lr_final."""
    import torch
    rng = np.random.default_rng(seed)
    log = TrainLog()
    t0 = time.perf_counter()
    for s in range(steps):
        p = pairs[int(rng.integers(len(pairs)))]
        cols = np.sort(rng.choice(p.R.shape[1], min(batch, p.R.shape[1]), replace=False))
        cols = torch.as_tensor(cols, device=p.R.device)
        R = p.R[:, cols].t().contiguous().t()
        E = p.E[:, cols].t().contiguous().t()
        lr_s = lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        loss = P.train_step(p.mesh, p.k, R, E, lr_s)
        if s % log_every == 0 or s == steps - 1:
            log.losses.append((s, float(loss)))
    log.seconds = time.perf_counter() - t0
    log.steps = steps
    return log


def evaluate(P, meshes, tol: float = 1e-6, ndirs: int = 4, seed: int = 996, restart: int = 100, maxit: int = 2000):
    """Plane-wave right-hand sides on each mesh, solved to tol (FP64 check)
    with flexible GMRES + network and with plain GMRES; iterations and times.
    The exact (FP64) residual judges both."""
    import torch
    rng = np.random.default_rng(seed)
    rows = []
    for mesh, k, meta in meshes:
        dirs = synth.plane_wave_dirs(rng, ndirs)
        F = g.rhs_planewave(mesh, k, dirs)
        res = {}
        for name, pre in (("gmres", None), ("fgmres_mpnn", P)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X, rep = g.gmres_solve(mesh, k, F, tol=tol, restart=restart, maxit=maxit, prec="auto", check_prec="fp64",
                                   max_refine=3, precond=pre)
            torch.cuda.synchronize()
            res[name] = dict(seconds=time.perf_counter() - t0, iterations=rep.iterations, status=rep.status,
                             fallback=rep.precond_fallback, true_residual=float(np.max(rep.true_residual)))
        rows.append(dict(level=meta["level"], nv=mesh.nv, k=k, **res))
    return rows
