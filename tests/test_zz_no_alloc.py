"""gyps_sl_apply_noalloc: the apply for callers that must not allocate device
memory while they run (their memory belongs to another allocator, or a
cudaMalloc and the synchronisation it can cause is not acceptable in their
loop).  Its scratch is a fixed array inside the library, shared by all calls.

Checked through the C ABI against gyps_sl_apply (FP32 far part, FP64
correction) and against the FP64 oracle on two calls in a row with different
inputs, so that a stale accumulator from the first call would show up in the
second; device memory in use does not change over repeated calls.  This file
is collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from parity import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP32_TOL = 1e-5  # relative, per column: the tolerance of the FP32 parity tests


def _colmajor(x):
    return torch.as_tensor(x).cuda().t().contiguous().t()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("level,q,k,nrhs", [(3, 7, 16.0, 1), (2, 3, 5.0, 3), (4, 3, 0.0, 2)])
def test_noalloc_matches_apply_two_calls(level, q, k, nrhs):
    import paper_1804_00995_gb300 as g
    lib = g.load()
    v, t = synth.icosphere(level)
    mesh = g.Mesh(v, t, q)
    om = oracle.Mesh(v, t, q)
    nv = mesh.nv
    for call in range(2):
        x = _colmajor(synth.random_complex(np.random.default_rng(100 * level + call), nv, nrhs))
        y_ref = torch.empty((nrhs, nv), dtype=torch.complex128, device="cuda").t()
        y_new = torch.full((nrhs, nv), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda").t()
        code = lib.gyps_sl_apply(mesh.handle, k, nrhs, x.data_ptr(), nv, y_ref.data_ptr(), nv,
                                 g.PREC["fp32"], 0, -1, -1, _stream())
        assert code == 0
        code = lib.gyps_sl_apply_noalloc(mesh.handle, k, nrhs, x.data_ptr(), nv, y_new.data_ptr(), nv, _stream())
        assert code == 0, g.GypsError(code, "").status
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel(a, b) < FP32_TOL, (call, rel(a, b))
        # and against the FP64 oracle on the same input
        assert rel(a, om.apply(k, x.cpu().numpy())) < FP32_TOL, call
        assert lib.gyps_mesh_check(mesh.handle, _stream()) == 0
    mesh.close()


def test_noalloc_allocates_no_device_memory():
    """After a first call (which looks up the scratch array's address), further
    calls leave the device's free memory unchanged."""
    import paper_1804_00995_gb300 as g
    lib = g.load()
    v, t = synth.icosphere(3)
    mesh = g.Mesh(v, t, 3)
    nv = mesh.nv
    x = _colmajor(synth.random_complex(np.random.default_rng(5), nv, 3))
    y = torch.empty((3, nv), dtype=torch.complex128, device="cuda").t()
    assert lib.gyps_sl_apply_noalloc(mesh.handle, 7.0, 3, x.data_ptr(), nv, y.data_ptr(), nv, _stream()) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert lib.gyps_sl_apply_noalloc(mesh.handle, 7.0, 3, x.data_ptr(), nv, y.data_ptr(), nv, _stream()) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    mesh.close()


def test_noalloc_rejects_host_buffers_and_oversized_meshes():
    import paper_1804_00995_gb300 as g
    lib = g.load()
    v, t = synth.icosphere(2)
    mesh = g.Mesh(v, t, 3)
    xh = np.zeros(mesh.nv, dtype=np.complex128)
    yh = np.zeros(mesh.nv, dtype=np.complex128)
    assert lib.gyps_sl_apply_noalloc(mesh.handle, 1.0, 1, xh.ctypes.data, mesh.nv, yh.ctypes.data, mesh.nv,
                                     _stream()) == 1
    mesh.close()
    # 573440 quadrature points need ~16 MB of scratch: beyond the fixed 8 MiB
    v, t = synth.icosphere(6)
    big = g.Mesh(v, t, 7)
    x = torch.zeros((big.nv, 1), dtype=torch.complex128, device="cuda")
    y = torch.zeros((big.nv, 1), dtype=torch.complex128, device="cuda")
    assert lib.gyps_sl_apply_noalloc(big.handle, 1.0, 1, x.data_ptr(), big.nv, y.data_ptr(), big.nv, _stream()) == 1
    buf = ctypes.create_string_buffer(512)
    lib.gyps_last_error(buf, 512)
    assert b"scratch" in buf.value
    big.close()
