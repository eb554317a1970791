"""Learned preconditioner on the GPU: the hand-written forward, backward and
Adam kernels against the FP64 oracle of the network; checkpointing; the
flexible-GMRES fallback when the network misbehaves; training lowers the loss."""
import numpy as np
import pytest

import synth
from oracle import mpnn as omp
from parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1804_00995_gb300 as g
    g.load()
    return g


def _setup(g, level=1, layers=4, seed=11, B=3):
    v, t = synth.ellipsoid(level, (0.8, 1.1, 1.5), (0.3, 1.0, 0.2), 0.9)
    mesh = g.Mesh(v, t, 3)
    P = g.Precond(64, layers, seed=seed)
    rng = np.random.default_rng(seed)
    R = synth.random_complex(rng, mesh.nv, B)
    E = synth.random_complex(rng, mesh.nv, B) * 50.0
    return v, t, mesh, P, R, E


def test_forward_matches_oracle(g):
    v, t, mesh, P, R, _ = _setup(g)
    p = P.get_params()
    # a non-trivial network: random weights (the initial decoder is small)
    rng = np.random.default_rng(2)
    p = (p + rng.normal(size=p.size).astype(np.float32) * 0.05).astype(np.float32)
    P.set_params(p)
    z = P.apply(mesh, 5.0, torch.as_tensor(R).cuda()).cpu().numpy()
    ref = omp.forward(p, v, t, 5.0, R, layers=4)
    assert rel(z, ref) < 1e-5


def test_gradient_matches_oracle(g):
    v, t, mesh, P, R, E = _setup(g, B=2)
    p = P.get_params()
    loss, grad = P.train_step(mesh, 7.0, torch.as_tensor(R).cuda(), torch.as_tensor(E).cuda(), 0.0, want_grad=True)
    lref, gref = omp.loss_and_grad(p, v, t, 7.0, R, E, layers=4)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    assert rel(grad, gref) < 1e-4
    # per block: every parameter group gets the right gradient
    off, _ = omp.layout(64, 4)
    for name, (o, shape) in off.items():
        n = int(np.prod(shape))
        if np.linalg.norm(gref[o:o + n]) > 1e-8 * np.linalg.norm(gref):
            assert rel(grad[o:o + n], gref[o:o + n]) < 1e-3, name


def test_adam_step_matches_formula(g):
    v, t, mesh, P, R, E = _setup(g, B=2)
    p0 = P.get_params().astype(np.float64)
    _, grad = P.train_step(mesh, 3.0, torch.as_tensor(R).cuda(), torch.as_tensor(E).cuda(), 0.0, want_grad=True)
    P.train_step(mesh, 3.0, torch.as_tensor(R).cuda(), torch.as_tensor(E).cuda(), 1e-3)
    p1 = P.get_params().astype(np.float64)
    pref, _, _ = omp.adam_step(p0, grad.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    assert np.abs(p1 - pref).max() < 1e-6
    assert P.steps() == 1


def test_checkpoint_round_trip_and_corrupt_file(g, tmp_path):
    v, t, mesh, P, R, E = _setup(g)
    for _ in range(3):
        P.train_step(mesh, 3.0, torch.as_tensor(R).cuda(), torch.as_tensor(E).cuda(), 1e-3)
    path = tmp_path / "net.bin"
    P.save(path)
    Q = g.Precond(64, 4, seed=99)
    Q.load(path)
    assert np.array_equal(Q.get_params(), P.get_params()) and Q.steps() == 3
    # a parameter corrupted on the host is refused, the network keeps its weights
    raw = bytearray(open(path, "rb").read())
    raw[256:260] = np.array([np.nan], dtype=np.float32).tobytes()
    bad = tmp_path / "bad.bin"
    open(bad, "wb").write(bytes(raw))
    before = Q.get_params()
    with pytest.raises(g.GypsError) as e:
        Q.load(bad)
    assert e.value.status == "NAN"
    assert np.array_equal(Q.get_params(), before)
    with pytest.raises(g.GypsError):
        g.Precond(64, 3, seed=1).load(path)  # other shape


def test_fgmres_falls_back_when_the_network_fails(g):
    """A network whose weights were poisoned on the host (a NaN) makes the
    first flexible cycle non-finite: the solver drops it and converges."""
    v, t = synth.icosphere(2)
    mesh = g.Mesh(v, t, 3)
    P = g.Precond(64, 4, seed=5)
    p = P.get_params()
    off, _ = omp.layout(64, 4)
    p[off["b_out"][0]] = np.nan  # the decoder bias reaches every output
    P.set_params(p)
    f = g.rhs_planewave(mesh, 4.0, [(0.0, 0.0, 1.0)])
    x, rep = g.gmres_solve(mesh, 4.0, f, tol=1e-6, restart=50, prec="fp32", check_prec="fp64", precond=P)
    assert rep.status == "OK" and rep.precond_fallback == 1 and rep.true_residual[0] <= 1e-6
    x0, rep0 = g.gmres_solve(mesh, 4.0, f, tol=1e-6, restart=50, prec="fp32", check_prec="fp64")
    assert np.linalg.norm((x - x0).cpu().numpy()) / np.linalg.norm(x0.cpu().numpy()) < 1e-4


def test_untrained_network_is_dropped_for_slow_progress(g):
    """An untrained network slows flexible GMRES down; the first cycle that does
    not halve the residual drops it and plain GMRES finishes."""
    v, t = synth.icosphere(2)
    mesh = g.Mesh(v, t, 3)
    P = g.Precond(64, 4, seed=5)
    f = g.rhs_planewave(mesh, 4.0, [(0.0, 0.0, 1.0)])
    x, rep = g.gmres_solve(mesh, 4.0, f, tol=1e-6, restart=30, prec="fp32", check_prec="fp64", precond=P)
    assert rep.status == "OK" and rep.true_residual[0] <= 1e-6
    assert rep.iterations < 200


def test_training_lowers_the_loss_and_fgmres_converges(g):
    """Train on correction pairs the solver generates (non-resonant k), then
    compare flexible GMRES + network with plain GMRES on held-out meshes: both
    reach the exact-residual tolerance, and the network saves iterations."""
    from paper_1804_00995_gb300 import precond_train as pt
    meshes = pt.random_meshes(995, 6, levels=(3,), k_range=(2.0, 4.0))
    pairs, stats = pt.make_pairs(meshes, nrhs=16, tol=1e-3, seed=1, k_range=(2.0, 4.0))
    assert len(pairs) >= 4, stats
    P = g.Precond(64, 4, seed=995)
    first = np.mean([P.train_step(p.mesh, p.k, p.R, p.E, 0.0) for p in pairs])
    pt.train(P, pairs, steps=600, lr=2e-3, batch=16, seed=2, lr_final=4e-4)
    last = np.mean([P.train_step(p.mesh, p.k, p.R, p.E, 0.0) for p in pairs])
    assert last < 0.5 * first, (first, last)
    test = pt.random_meshes(996, 2, levels=(3,), k_range=(2.0, 4.0))
    rows = pt.evaluate(P, test, tol=1e-6, ndirs=2, restart=30)
    for r in rows:
        assert r["gmres"]["status"] == "OK" and r["fgmres_mpnn"]["status"] == "OK", r
        assert r["fgmres_mpnn"]["true_residual"] <= 1e-6
    assert sum(r["fgmres_mpnn"]["iterations"] for r in rows) < sum(r["gmres"]["iterations"] for r in rows), rows
    kept = [r for r in rows if r["fgmres_mpnn"]["fallback"] == 0]
    assert kept, rows
    print([(r["gmres"]["iterations"], r["fgmres_mpnn"]["iterations"], round(r["gmres"]["seconds"], 4),
            round(r["fgmres_mpnn"]["seconds"], 4)) for r in rows])
    # where the network is kept it also saves wall time (iterations cost more with it)
    assert sum(r["fgmres_mpnn"]["seconds"] for r in kept) < sum(r["gmres"]["seconds"] for r in kept), rows


def test_krylov_pairs_are_exact_and_follow_the_gmres_residuals(g):
    """Krylov training pairs: each residual R_m is V applied to the error
    E_m = X* - X_m of the m-step GMRES iterate (checked against the oracle's
    dense V element by element), and the residual norms fall with m as GMRES
    minimises them; training on the pairs lowers the loss."""
    import oracle
    from paper_1804_00995_gb300 import precond_train as pt
    meshes = pt.random_meshes(997, 1, levels=(2,), k_range=(1.0, 1.4))  # below the first interior resonance
    steps = (2, 5, 10)
    # tol above the FP32 check's floor (the solves' converged flags come from that check)
    pairs, stats = pt.make_krylov_pairs(meshes, ndirs=3, steps=steps, tol=1e-6, maxit=400, seed=4)
    assert len(pairs) == 1 and stats[0]["kept"] == 3 * len(steps), stats
    p = pairs[0]
    meta = meshes[0][2]
    V = oracle.Mesh(meta["vtx"], meta["tri"], 3).assemble(p.k)
    E = p.E.cpu().numpy()
    R = p.R.cpu().numpy()
    ref = V @ E
    tol = 1e-5  # FP32 far part of the apply
    for c in range(R.shape[1]):
        assert np.abs(R[:, c] - ref[:, c]).max() <= tol * np.abs(ref[:, c]).max(), c
    norms = np.linalg.norm(R, axis=0).reshape(len(steps), 3)
    assert np.all(norms[1:] <= norms[:-1] * (1 + 1e-4)), norms
    assert np.all(norms[-1] < 0.5 * norms[0]), norms
    P = g.Precond(64, 4, seed=7)
    first = P.train_step(p.mesh, p.k, p.R, p.E, 0.0)
    pt.train(P, pairs, steps=200, lr=2e-3, batch=9, seed=2, lr_final=4e-4)
    last = P.train_step(p.mesh, p.k, p.R, p.E, 0.0)
    assert last < 0.5 * first, (first, last)


def test_network_is_used_only_inside_its_training_range(g, tmp_path):
    """The network records the electrical sizes k x radius it was trained on;
    flexible GMRES leaves it out (fallback 2, plain GMRES iterations) for a
    mesh and k outside that range widened by 25 %, and uses it inside; the
    range survives a checkpoint."""
    v, t = synth.icosphere(2)
    mesh = g.Mesh(v, t, 3)
    P = g.Precond(64, 4, seed=5)
    lo, hi = P.range()
    assert lo > hi  # untrained: no range
    rng = np.random.default_rng(5)
    R = torch.as_tensor(synth.random_complex(rng, mesh.nv, 4)).cuda()
    P.train_step(mesh, 3.0, R, R, 0.0)  # lr = 0: the gradient only, the range is recorded
    lo, hi = P.range()
    assert abs(lo - 3.0) < 1e-6 and abs(hi - 3.0) < 1e-6  # unit sphere: radius 1
    path = str(tmp_path / "p.bin")
    P.save(path)
    Q = g.Precond(64, 4, seed=6)
    Q.load(path)
    assert Q.range() == (lo, hi)
    F = g.rhs_planewave(mesh, 9.0, [(0.0, 0.0, 1.0)])
    x0, r0 = g.gmres_solve(mesh, 9.0, F, tol=1e-6, restart=100, prec="fp32", check_prec="df64")
    x1, r1 = g.gmres_solve(mesh, 9.0, F, tol=1e-6, restart=100, prec="fp32", check_prec="df64", precond=Q)
    assert r1.precond_fallback == 2 and r1.iterations == r0.iterations and r1.status == "OK"
    F3 = g.rhs_planewave(mesh, 3.3, [(0.0, 0.0, 1.0)])
    _, r2 = g.gmres_solve(mesh, 3.3, F3, tol=1e-6, restart=100, prec="fp32", check_prec="df64", precond=Q)
    assert r2.precond_fallback != 2
