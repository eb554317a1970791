"""Pins of the FP64 oracle of the preconditioner network: gradient by central
finite differences, equivariances the definition implies, bf16 rounding."""
import numpy as np
import pytest

import synth
from oracle import mpnn


def _params(seed, hidden=64, layers=2):
    _, n = mpnn.layout(hidden, layers)
    rng = np.random.default_rng(seed)
    return (rng.normal(size=n) * 0.2).astype(np.float32)


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8, 3.0e-39],
                 dtype=np.float32)
    got = mpnn.bf16_round(x)
    # halfway cases round to the even mantissa; 3e-39 is subnormal in float32
    exp = [1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.0 + 2.0 ** -6, None]
    for g, e in zip(got[:5], exp[:5]):
        assert g == e
    assert abs(got[5] - 3.0e-39) < 1e-40


def test_gradient_matches_central_differences():
    v, t = synth.icosphere(0)
    rng = np.random.default_rng(3)
    R = synth.random_complex(rng, v.shape[0], 2)
    E = synth.random_complex(rng, v.shape[0], 2) * 30.0
    p = _params(1)
    loss, g = mpnn.loss_and_grad(p, v, t, 2.5, R, E, layers=2)
    w = mpnn.bf16_round(p)
    assert abs(loss - mpnn.loss_from_rounded(w, v, t, 2.5, R, E, layers=2)) < 1e-12
    idx = rng.choice(w.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mpnn.loss_from_rounded(wp, v, t, 2.5, R, E, layers=2) -
              mpnn.loss_from_rounded(wm, v, t, 2.5, R, E, layers=2)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_output_scales_with_the_residual():
    """M(a r) = a M(r) for a > 0: inputs are normalised by rms(r), outputs rescaled by it."""
    v, t = synth.icosphere(1)
    R = synth.random_complex(np.random.default_rng(5), v.shape[0], 1)
    p = _params(2)
    z1 = mpnn.forward(p, v, t, 4.0, R, layers=2)
    z2 = mpnn.forward(p, v, t, 4.0, 7.5 * R, layers=2)
    assert np.abs(z2 - 7.5 * z1).max() <= 1e-12 * np.abs(z2).max()


def test_vertex_relabelling_permutes_the_output():
    v, t = synth.icosphere(1)
    nv = v.shape[0]
    perm = np.random.default_rng(6).permutation(nv)
    inv = np.argsort(perm)
    v2 = v[perm]
    t2 = inv[t].astype(np.int32)
    R = synth.random_complex(np.random.default_rng(7), nv, 1)
    p = _params(3)
    z = mpnn.forward(p, v, t, 6.0, R, layers=2)
    z2 = mpnn.forward(p, v2, t2, 6.0, R[perm], layers=2)
    assert np.abs(z2 - z[perm]).max() <= 1e-11 * np.abs(z).max()


def test_adam_matches_hand_computation():
    p = np.array([1.0, -2.0]); g = np.array([0.5, -0.25]); m = np.zeros(2); v = np.zeros(2)
    p1, m1, v1 = mpnn.adam_step(p, g, m, v, 1, 0.1)
    # first step: m^ = g, v^ = g^2 -> p - lr * sign(g) (up to eps)
    assert np.allclose(p1, p - 0.1 * np.sign(g), atol=1e-6)
