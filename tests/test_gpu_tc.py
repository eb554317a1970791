"""Tensor-core form of the kernel product (bf16 hi+lo split, three products,
FP32 accumulation in tensor memory) against the FP64 oracle and the FP32
CUDA-core apply.  Tolerance 1e-4 relative per column (split bf16 products)."""
import numpy as np
import pytest

import oracle
import synth
from parity import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TC_TOL = 1e-4


@pytest.mark.parametrize("level,q,k,nrhs", [(1, 3, 5.0, 16), (2, 3, 16.0, 16), (2, 7, 9.0, 20), (3, 3, 30.0, 32), (3, 3, 12.0, 64), (2, 7, 7.0, 70)])
def test_tc_apply_vs_oracle(level, q, k, nrhs):
    import paper_1804_00995_gb300 as g
    v, t = synth.icosphere(level)
    gm = g.Mesh(v, t, q)
    om = oracle.Mesh(v, t, q)
    x = synth.random_complex(np.random.default_rng(level * 10 + nrhs), om.nv, nrhs)
    xd = torch.as_tensor(x).cuda()
    y = g.sl_apply(gm, k, xd, prec="tc_bf16x3").cpu().numpy()
    assert np.isfinite(y).all()
    ref = om.apply(k, x)
    assert rel(y, ref) < TC_TOL
    y32 = g.sl_apply(gm, k, xd, prec="fp32").cpu().numpy()
    assert rel(y, y32) < TC_TOL
    # auto picks the tensor cores at nrhs >= 16
    ya = g.sl_apply(gm, k, xd, prec="auto").cpu().numpy()
    assert rel(ya, y) < 1e-12


def test_tc_far_part_ellipsoid():
    import paper_1804_00995_gb300 as g
    v, t = synth.ellipsoid(2, (0.6, 1.4, 1.9), (1.0, -1.0, 0.3), 1.1)
    gm = g.Mesh(v, t, 3)
    om = oracle.Mesh(v, t, 3)
    x = synth.random_complex(np.random.default_rng(4), om.nv, 16)
    y = g.sl_apply(gm, 11.0, torch.as_tensor(x).cuda(), prec="tc_bf16x3", near=False).cpu().numpy()
    assert rel(y, om.far_apply(11.0, x)) < TC_TOL


def test_tc_rejects_laplace():
    import paper_1804_00995_gb300 as g
    v, t = synth.icosphere(1)
    gm = g.Mesh(v, t, 3)
    x = torch.zeros((gm.nv, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.GypsError) as e:
        g.sl_apply(gm, 0.0, x, prec="tc_bf16x3")
    assert e.value.status == "UNSUPPORTED"


@pytest.mark.parametrize("nrhs", [16, 40])
def test_tc_triangle_ranges_add_up(nrhs):
    """Tensor-core applies over a partition of the test triangles (ragged cuts,
    one range of a single triangle) sum to the full tensor-core apply, and each
    partial apply matches the oracle's rows of that range."""
    import paper_1804_00995_gb300 as g
    v, t = synth.icosphere(3)
    gm = g.Mesh(v, t, 3)
    om = oracle.Mesh(v, t, 3)
    x = synth.random_complex(np.random.default_rng(nrhs), om.nv, nrhs)
    xd = torch.as_tensor(x).cuda()
    full = g.sl_apply(gm, 9.0, xd, prec="tc_bf16x3").cpu().numpy()
    cuts = [0, 300, 301, 777, om.nt]
    parts = [g.sl_apply(gm, 9.0, xd, prec="tc_bf16x3", tri_range=(a, b)).cpu().numpy() for a, b in zip(cuts[:-1], cuts[1:])]
    assert rel(sum(parts), full) < 1e-6
    assert rel(full, om.apply(9.0, x)) < TC_TOL
    empty = g.sl_apply(gm, 9.0, xd, prec="tc_bf16x3", tri_range=(5, 5)).cpu().numpy()
    assert np.abs(empty).max() == 0.0


@pytest.mark.slow
def test_sphere163842_k64_q3_r16_sampled_rows():
    """Workload sphere163842_k64_q3_r16 at full size (983040 points, 16 plane
    waves, seed 7): tensor-core apply (16 columns) and the FP32 CUDA-core apply
    (2 columns) vs the oracle on 48 sampled rows."""
    import paper_1804_00995_gb300 as g
    v, t = synth.icosphere(7)
    gm = g.Mesh(v, t, 3)
    om = oracle.Mesh(v, t, 3)
    dirs = synth.plane_wave_dirs(np.random.default_rng(7), 16)
    f = g.rhs_planewave(gm, 64.0, dirs)
    y = g.sl_apply(gm, 64.0, f, prec="tc_bf16x3").cpu().numpy()
    fh = f.cpu().numpy()
    rows = np.sort(np.random.default_rng(64).choice(om.nv, 48, replace=False))
    ref = om.apply(64.0, fh, rows=rows)[rows]
    assert rel(y[rows], ref) < TC_TOL
    # the FP32 CUDA-core form at the same k (phases up to about 130 rad), two columns
    y32 = g.sl_apply(gm, 64.0, f[:, :2], prec="fp32").cpu().numpy()
    assert rel(y32[rows], ref[:, :2]) < 1e-5
