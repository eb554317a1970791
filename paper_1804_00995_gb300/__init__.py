"""Python binding of libgyps (GB300 Galerkin Helmholtz single layer on P1 meshes).

Argument marshalling only: every step of the operator runs in the CUDA kernels
of ``libgyps.so``, behind the C ABI declared in ``include/gyps.h``.  Torch is
used for device memory and streams.  Importing works without the library; the
first call that needs it raises ``RuntimeError`` when it has not been built
(``python -m paper_1804_00995_gb300.build``).

Complex blocks are torch ``complex128`` tensors of shape (nv,) or (nv, nrhs);
they are passed column-major (stride (1, ld)), copied to that layout when
needed.  CPU tensors are accepted too: the library then stages them through
device memory and the call returns when the result is back on the host.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "PREC", "GypsError", "Mesh", "load", "sl_apply", "near_correct", "sl_assemble", "rhs_planewave",
    "gmres_solve", "version", "set_wait_polls", "Hmat",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgyps.so")

PREC = {"fp64": 0, "fp32": 1, "tc_bf16x3": 2, "df64": 3, "auto": 4, "hmat": 5}
NO_NEAR = 0x1

_STATUS = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "NAN", 6: "TIMEOUT", 7: "UNSUPPORTED"}


class GypsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gyps {_STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = _STATUS.get(code, str(code))


class _MeshInfo(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nt", ctypes.c_int64), ("nq", ctypes.c_int64), ("q", ctypes.c_int32),
                ("device", ctypes.c_int32), ("near_pairs", ctypes.c_int64), ("near_nnz", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class _Profile(ctypes.Structure):
    _fields_ = [("applies", ctypes.c_int64), ("launches", ctypes.c_int64), ("interp_ms", ctypes.c_double),
                ("far_ms", ctypes.c_double), ("project_ms", ctypes.c_double), ("near_ms", ctypes.c_double),
                ("far_launches", ctypes.c_int64)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("k", ctypes.c_double), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64),
                ("Y", ctypes.c_void_p), ("ldy", ctypes.c_int64)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("nmesh", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("rhs_chunk", ctypes.c_int32),
                ("targets_per_thread", ctypes.c_int32), ("grid", ctypes.c_int32), ("uses_graph", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("tensor_cores", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("work_items", ctypes.c_int64), ("pairs", ctypes.c_double)]


class _HmatInfo(ctypes.Structure):
    _fields_ = [("clusters", ctypes.c_int64), ("dense_blocks", ctypes.c_int64), ("lowrank_blocks", ctypes.c_int64),
                ("fallback_blocks", ctypes.c_int64), ("max_rank", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mean_rank", ctypes.c_double), ("bytes", ctypes.c_int64), ("dense_bytes", ctypes.c_double),
                ("build_ms", ctypes.c_double)]


class _GmresOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("check_prec", ctypes.c_int32), ("use_x0", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("precond", ctypes.c_void_p), ("formulation", ctypes.c_int32),
                ("eta", ctypes.c_double), ("timeout_ms", ctypes.c_double), ("hmat", ctypes.c_void_p)]


class _GmresReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("applies", ctypes.c_int32), ("check_applies", ctypes.c_int32),
                ("refinements", ctypes.c_int32), ("precond_fallback", ctypes.c_int32),
                ("est_residual", ctypes.POINTER(ctypes.c_double)),
                ("true_residual", ctypes.POINTER(ctypes.c_double)), ("converged", ctypes.POINTER(ctypes.c_int32))]


_lib = None

# every symbol the header declares, with its ctypes signature
_SIGS = {
    "gyps_version": ([], ctypes.c_char_p),
    "gyps_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "gyps_mesh_create": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                          ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "gyps_mesh_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "gyps_mesh_info": ([ctypes.c_void_p, ctypes.POINTER(_MeshInfo)], ctypes.c_int),
    "gyps_quad_points": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "gyps_near_export": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "gyps_sl_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_int64,
                       ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_near_correct": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_sl_assemble": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                          ctypes.c_void_p], ctypes.c_int),
    "gyps_dl_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_adl_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_cfie_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_rhs_planewave_cfie": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_rwg_edges": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_void_p],
                       ctypes.c_int),
    "gyps_efie_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_rhs_planewave_efie": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_mfie_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_emcfie_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_rhs_planewave_emcfie": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_bw_apply": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "gyps_sl_potential": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p],
                          ctypes.c_int),
    "gyps_rhs_planewave": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_gmres_solve": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                          ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(_GmresOpts),
                          ctypes.POINTER(_GmresReport), ctypes.c_void_p], ctypes.c_int),
    "gyps_batch_create": ([ctypes.POINTER(_BatchItem), ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "gyps_batch_apply": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "gyps_batch_info": ([ctypes.c_void_p, ctypes.POINTER(_BatchInfo)], ctypes.c_int),
    "gyps_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "gyps_mesh_check": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "gyps_hmat_create": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "gyps_hmat_apply": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                         ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_hmat_info": ([ctypes.c_void_p, ctypes.POINTER(_HmatInfo)], ctypes.c_int),
    "gyps_hmat_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "gyps_set_wait_polls": ([ctypes.c_int64], ctypes.c_int),
    "gyps_sl_apply_noalloc": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_precond_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)],
                            ctypes.c_int),
    "gyps_precond_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "gyps_precond_range": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                           ctypes.c_int),
    "gyps_precond_info": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "gyps_precond_params": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
    "gyps_precond_apply": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "gyps_precond_train_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "gyps_precond_save": ([ctypes.c_void_p, ctypes.c_char_p], ctypes.c_int),
    "gyps_precond_load": ([ctypes.c_void_p, ctypes.c_char_p], ctypes.c_int),
    "gyps_profile_enable": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "gyps_profile_read": ([ctypes.c_void_p, ctypes.POINTER(_Profile)], ctypes.c_int),
}


def load(path: str = LIB_PATH):
    """Loads libgyps.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libgyps.so not built at {path}: run python -m paper_1804_00995_gb300.build")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def version() -> str:
    return load().gyps_version().decode()


def _check(code):
    if code != 0:
        buf = ctypes.create_string_buffer(512)
        load().gyps_last_error(buf, 512)
        raise GypsError(code, buf.value.decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _colmajor(x, nv, name):
    """Returns (tensor, nrhs, ld) with x viewed column-major complex128."""
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(np.asarray(x))
    if x.dtype != torch.complex128:
        x = x.to(torch.complex128)
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    if x.dim() != 2 or x.shape[0] != nv:
        raise ValueError(f"{name} must have shape (nv,) or (nv, nrhs) with nv={nv}")
    if x.stride(0) != 1 or x.stride(1) < nv:
        x = x.t().contiguous().t()
    return x, x.shape[1], max(x.stride(1), nv) if x.shape[1] > 1 else nv


def _empty_colmajor(nv, nrhs, device):
    torch = _torch()
    return torch.empty((nrhs, nv), dtype=torch.complex128, device=device).t()


@dataclass
class MeshInfo:
    nv: int
    nt: int
    nq: int
    q: int
    device: int
    near_pairs: int
    near_nnz: int
    device_bytes: int


class Mesh:
    """gyps_mesh_create: mesh, Gauss rule dom(mesh, q), P1 space and the correction C."""

    def __init__(self, vtx, tri, q: int = 3, stream=None):
        lib = load()
        vtx = np.ascontiguousarray(np.asarray(vtx, dtype=np.float64))
        tri = np.ascontiguousarray(np.asarray(tri, dtype=np.int32))
        if vtx.ndim != 2 or vtx.shape[1] != 3 or tri.ndim != 2 or tri.shape[1] != 3:
            raise ValueError("vtx must be (nv, 3) and tri (nt, 3)")
        h = ctypes.c_void_p()
        _check(lib.gyps_mesh_create(vtx.ctypes.data, vtx.shape[0], tri.ctypes.data, tri.shape[0], int(q), 0,
                                    _stream(stream), ctypes.byref(h)))
        self._h = h
        info = _MeshInfo()
        _check(lib.gyps_mesh_info(self._h, ctypes.byref(info)))
        self.info = MeshInfo(info.nv, info.nt, info.nq, info.q, info.device, info.near_pairs, info.near_nnz,
                             info.device_bytes)
        self.nv, self.nt, self.nq, self.q = info.nv, info.nt, info.nq, info.q
        self.device = f"cuda:{info.device}"

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("mesh was closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.gyps_mesh_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def quad_points(self, stream=None):
        """(nq, 4) float64 tensor (x, y, z, w) on the mesh's device."""
        torch = _torch()
        out = torch.empty((self.nq, 4), dtype=torch.float64, device=self.device)
        _check(load().gyps_quad_points(self.handle, out.data_ptr(), _stream(stream)))
        return out

    def profile(self, enable: bool = True):
        """Turns per-stage device timing of sl_apply on or off (resets totals)."""
        _check(load().gyps_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self) -> dict:
        """Totals since profiling was enabled: applies, launches, per-stage ms."""
        p = _Profile()
        _check(load().gyps_profile_read(self.handle, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in _Profile._fields_}

    def check(self, stream=None):
        """Synchronises the stream, then reads and clears the error word of the
        mesh's bounded device waits (gyps_mesh_check); raises GypsError
        (TIMEOUT) if a wait of an asynchronous call gave up."""
        _check(load().gyps_mesh_check(self.handle, _stream(stream)))

    def near_csr(self):
        """Correction matrix C (CSR: rowptr int64, col int32, val float64), host numpy."""
        rowptr = np.zeros(self.nv + 1, dtype=np.int64)
        col = np.zeros(self.info.near_nnz, dtype=np.int32)
        val = np.zeros(self.info.near_nnz, dtype=np.float64)
        _check(load().gyps_near_export(self.handle, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rowptr, col, val


def set_wait_polls(polls: int) -> None:
    """Poll limit of the far kernels' pipeline waits, process-wide
    (gyps_set_wait_polls): negative restores the defaults, 0 makes every such
    wait give up at once (tests of the TIMEOUT path)."""
    _check(load().gyps_set_wait_polls(int(polls)))


def sl_apply(mesh: Mesh, k: float, X, prec: str = "fp32", near: bool = True, tri_range=None, out=None, stream=None):
    """Y = (1/4pi) Phi^T W G W Phi X + C X (gyps_sl_apply).  Returns Y shaped like X."""
    torch = _torch()
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, mesh.nv, "X")
    y = out if out is not None else _empty_colmajor(mesh.nv, nrhs, x.device)
    if y.stride(0) != 1:
        raise ValueError("out must be column-major")
    tb, te = (-1, -1) if tri_range is None else (int(tri_range[0]), int(tri_range[1]))
    _check(load().gyps_sl_apply(mesh.handle, float(k), nrhs, x.data_ptr(), ldx, y.data_ptr(),
                                max(y.stride(1), mesh.nv) if nrhs > 1 else mesh.nv, PREC[prec],
                                0 if near else NO_NEAR, tb, te, _stream(stream)))
    return y[:, 0] if one else y


def near_correct(mesh: Mesh, X, Y, stream=None):
    """Y += C X in place (gyps_near_correct); Y column-major complex128."""
    x, nrhs, ldx = _colmajor(X, mesh.nv, "X")
    y = Y.reshape(-1, 1) if Y.dim() == 1 else Y
    if y.stride(0) != 1 or y.dtype != _torch().complex128:
        raise ValueError("Y must be column-major complex128")
    _check(load().gyps_near_correct(mesh.handle, nrhs, x.data_ptr(), ldx, y.data_ptr(),
                                    max(y.stride(1), mesh.nv) if nrhs > 1 else mesh.nv, _stream(stream)))
    return Y


def sl_assemble(mesh: Mesh, k: float, prec: str = "fp64", device=None, out=None, stream=None):
    """Dense V (nv, nv) complex128, column-major, V[i, j] = test i, trial j (gyps_sl_assemble).
    out: a column-major (nv, nv) complex128 tensor to assemble into."""
    if out is None:
        dev = mesh.device if device is None else device
        out = _empty_colmajor(mesh.nv, mesh.nv, dev)
    elif out.stride(0) != 1 or tuple(out.shape) != (mesh.nv, mesh.nv):
        raise ValueError("out must be a column-major (nv, nv) tensor")
    _check(load().gyps_sl_assemble(mesh.handle, float(k), PREC[prec], out.data_ptr(), max(out.stride(1), mesh.nv),
                                   _stream(stream)))
    return out


def dl_apply(mesh: Mesh, k: float, X, prec: str = "fp32", stream=None):
    """Y = K X, the Galerkin double layer with its 'grady[1/r]' correction (gyps_dl_apply)."""
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, mesh.nv, "X")
    y = _empty_colmajor(mesh.nv, nrhs, x.device)
    _check(load().gyps_dl_apply(mesh.handle, float(k), nrhs, x.data_ptr(), ldx, y.data_ptr(),
                                max(y.stride(1), mesh.nv) if nrhs > 1 else mesh.nv, PREC[prec], _stream(stream)))
    return y[:, 0] if one else y


def adl_apply(mesh: Mesh, k: float, X, prec: str = "fp32", stream=None):
    """Y = K' X, the Galerkin adjoint double layer (gyps_adl_apply)."""
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, mesh.nv, "X")
    y = _empty_colmajor(mesh.nv, nrhs, x.device)
    _check(load().gyps_adl_apply(mesh.handle, float(k), nrhs, x.data_ptr(), ldx, y.data_ptr(),
                                 max(y.stride(1), mesh.nv) if nrhs > 1 else mesh.nv, PREC[prec], _stream(stream)))
    return y[:, 0] if one else y


def _combined(fn, mesh, k, eta, X, prec, stream):
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, mesh.nv, "X")
    y = _empty_colmajor(mesh.nv, nrhs, x.device)
    _check(fn(mesh.handle, float(k), float(eta), nrhs, x.data_ptr(), ldx, y.data_ptr(),
              max(y.stride(1), mesh.nv) if nrhs > 1 else mesh.nv, PREC[prec], _stream(stream)))
    return y[:, 0] if one else y


def bw_apply(mesh: Mesh, k: float, eta: float, X, prec: str = "fp32", stream=None):
    """Y = (1/2 M + K - i eta V) X, the Brakhage-Werner combined operator (gyps_bw_apply)."""
    return _combined(load().gyps_bw_apply, mesh, k, eta, X, prec, stream)


def cfie_apply(mesh: Mesh, k: float, eta: float, X, prec: str = "fp32", stream=None):
    """Y = (1/2 M + K' - i eta V) X, the direct combined-field operator (gyps_cfie_apply)."""
    return _combined(load().gyps_cfie_apply, mesh, k, eta, X, prec, stream)


def sl_potential(mesh: Mesh, k: float, pts, X, prec: str = "fp32", stream=None):
    """P (npts, nrhs): the single-layer potential of the density X at the points
    pts (npts, 3), with the [1/r] regularisation near the surface (gyps_sl_potential).
    pts and X on the device give P on the device; host inputs give host output."""
    torch = _torch()
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, mesh.nv, "X")
    if hasattr(pts, "dim"):
        p = pts.to(torch.float64).contiguous()
    else:
        p = torch.as_tensor(np.ascontiguousarray(np.asarray(pts, dtype=np.float64)))
    if p.dim() != 2 or p.shape[1] != 3:
        raise ValueError("pts must be (npts, 3)")
    npts = p.shape[0]
    out = _empty_colmajor(max(npts, 1), nrhs, x.device)[:npts]
    ldp = max(npts, 1)
    _check(load().gyps_sl_potential(mesh.handle, float(k), npts, p.data_ptr(), nrhs, x.data_ptr(), ldx,
                                    out.data_ptr(), ldp, PREC[prec], _stream(stream)))
    return out[:, 0] if one else out


def rhs_planewave(mesh: Mesh, k: float, dirs, device=None, stream=None):
    """F (nv, nrhs): F_ij = int phi_i exp(i k d_j . x) (gyps_rhs_planewave)."""
    dirs = np.ascontiguousarray(np.atleast_2d(np.asarray(dirs, dtype=np.float64)))
    dev = mesh.device if device is None else device
    f = _empty_colmajor(mesh.nv, dirs.shape[0], dev)
    _check(load().gyps_rhs_planewave(mesh.handle, float(k), dirs.shape[0], dirs.ctypes.data, f.data_ptr(), mesh.nv,
                                     _stream(stream)))
    return f


def rwg_edges(mesh: Mesh, stream=None):
    """(ne, edges (ne, 2) int32 vertex pairs): the RWG functions of the mesh (gyps_rwg_edges)."""
    ne = ctypes.c_int64()
    _check(load().gyps_rwg_edges(mesh.handle, ctypes.byref(ne), None, _stream(stream)))
    edges = np.zeros((ne.value, 2), dtype=np.int32)
    _check(load().gyps_rwg_edges(mesh.handle, ctypes.byref(ne), edges.ctypes.data, _stream(stream)))
    return ne.value, edges


def efie_apply(mesh: Mesh, k: float, X, prec: str = "fp32", stream=None):
    """Y = T X, the EFIE operator on the RWG coefficients (gyps_efie_apply); X: (ne,) or (ne, nrhs)."""
    ne, _ = rwg_edges(mesh, stream)
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, ne, "X")
    y = _empty_colmajor(ne, nrhs, x.device)
    _check(load().gyps_efie_apply(mesh.handle, float(k), nrhs, x.data_ptr(), ldx, y.data_ptr(),
                                  max(y.stride(1), ne) if nrhs > 1 else ne, PREC[prec], _stream(stream)))
    return y[:, 0] if one else y


def _em_apply(mesh, fn, args, X, stream):
    ne, _ = rwg_edges(mesh, stream)
    one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
    x, nrhs, ldx = _colmajor(X, ne, "X")
    y = _empty_colmajor(ne, nrhs, x.device)
    _check(fn(mesh.handle, *args[:-1], nrhs, x.data_ptr(), ldx, y.data_ptr(), max(y.stride(1), ne) if nrhs > 1 else ne,
              args[-1], _stream(stream)))
    return y[:, 0] if one else y


def mfie_apply(mesh: Mesh, k: float, X, prec: str = "fp32", stream=None):
    """Y = nxK X, the MFIE part of the electromagnetic listing (gyps_mfie_apply)."""
    return _em_apply(mesh, load().gyps_mfie_apply, (float(k), PREC[prec]), X, stream)


def emcfie_apply(mesh: Mesh, k: float, beta: float, X, prec: str = "fp32", stream=None):
    """Y = (-beta T + (1 - beta)(Id/2 - nxK)) X, the listing's LHS (gyps_emcfie_apply)."""
    return _em_apply(mesh, load().gyps_emcfie_apply, (float(k), float(beta), PREC[prec]), X, stream)


def rhs_planewave_emcfie(mesh: Mesh, k: float, beta: float, dirs, pols, device=None, stream=None):
    """F (ne, nrhs): beta int phi . E_inc - (1 - beta) int (n x phi) . H_inc (gyps_rhs_planewave_emcfie)."""
    ne, _ = rwg_edges(mesh, stream)
    dirs = np.ascontiguousarray(np.atleast_2d(np.asarray(dirs, dtype=np.float64)))
    pols = np.ascontiguousarray(np.atleast_2d(np.asarray(pols, dtype=np.float64)))
    if dirs.shape != pols.shape:
        raise ValueError("one polarisation per direction")
    dev = mesh.device if device is None else device
    f = _empty_colmajor(ne, dirs.shape[0], dev)
    _check(load().gyps_rhs_planewave_emcfie(mesh.handle, float(k), float(beta), dirs.shape[0], dirs.ctypes.data,
                                            pols.ctypes.data, f.data_ptr(), ne, _stream(stream)))
    return f


def rhs_planewave_efie(mesh: Mesh, k: float, dirs, pols, device=None, stream=None):
    """F (ne, nrhs): F_ej = int phi_e . p_j exp(i k d_j . x) (gyps_rhs_planewave_efie)."""
    ne, _ = rwg_edges(mesh, stream)
    dirs = np.ascontiguousarray(np.atleast_2d(np.asarray(dirs, dtype=np.float64)))
    pols = np.ascontiguousarray(np.atleast_2d(np.asarray(pols, dtype=np.float64)))
    if dirs.shape != pols.shape:
        raise ValueError("one polarisation per direction")
    dev = mesh.device if device is None else device
    f = _empty_colmajor(ne, dirs.shape[0], dev)
    _check(load().gyps_rhs_planewave_efie(mesh.handle, float(k), dirs.shape[0], dirs.ctypes.data, pols.ctypes.data,
                                          f.data_ptr(), ne, _stream(stream)))
    return f


def rhs_planewave_cfie(mesh: Mesh, k: float, eta: float, dirs, device=None, stream=None):
    """F (nv, nrhs): F_ij = int phi_i (d/dn - i eta) exp(i k d_j . x) (gyps_rhs_planewave_cfie)."""
    dirs = np.ascontiguousarray(np.atleast_2d(np.asarray(dirs, dtype=np.float64)))
    dev = mesh.device if device is None else device
    f = _empty_colmajor(mesh.nv, dirs.shape[0], dev)
    _check(load().gyps_rhs_planewave_cfie(mesh.handle, float(k), float(eta), dirs.shape[0], dirs.ctypes.data,
                                          f.data_ptr(), mesh.nv, _stream(stream)))
    return f


class Hmat:
    """Compressed far field of the single layer plus the correction
    (gyps_hmat_create / apply): Y = (H + C) X, H the block low-rank Gauss-Gauss
    part to relative tolerance eps."""

    def __init__(self, mesh: "Mesh", k: float, eps: float = 1e-5, leaf_tiles: int = 8, eta: float = 0.5,
                 stream=None):
        self.mesh = mesh
        self.k = float(k)
        h = ctypes.c_void_p()
        _check(load().gyps_hmat_create(mesh.handle, self.k, float(eps), int(leaf_tiles), float(eta), _stream(stream),
                                       ctypes.byref(h)))
        self._h = h

    @property
    def info(self) -> dict:
        i = _HmatInfo()
        _check(load().gyps_hmat_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _HmatInfo._fields_}

    def apply(self, X, out=None, stream=None):
        one = (hasattr(X, "dim") and X.dim() == 1) or (not hasattr(X, "dim") and np.asarray(X).ndim == 1)
        x, nrhs, ldx = _colmajor(X, self.mesh.nv, "X")
        y = out if out is not None else _empty_colmajor(self.mesh.nv, nrhs, x.device)
        if y.stride(0) != 1:
            raise ValueError("out must be column-major")
        _check(load().gyps_hmat_apply(self._h, nrhs, x.data_ptr(), ldx, y.data_ptr(),
                                      max(y.stride(1), self.mesh.nv) if nrhs > 1 else self.mesh.nv, _stream(stream)))
        return y[:, 0] if one else y

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            code = _lib.gyps_hmat_destroy(self._h)
            self._h = None
            _check(code)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """gyps_batch_create / apply: Y_i = V_i X_i for many meshes in one persistent launch.

    items: list of (mesh, k); X, Y are allocated here as column-major
    complex128 (nv_i, nrhs) device tensors (``self.X[i]``, ``self.Y[i]``) and
    bound to the batch: fill ``X[i]`` in place, call ``apply()``.
    """

    def __init__(self, items, nrhs: int, graph: bool = True, autotune: bool = False, cuda_cores: bool = False,
                 stream=None):
        torch = _torch()
        self.meshes = [m for m, _ in items]
        self.ks = [float(k) for _, k in items]
        self.X = [_empty_colmajor(m.nv, nrhs, m.device) for m in self.meshes]
        self.Y = [_empty_colmajor(m.nv, nrhs, m.device) for m in self.meshes]
        for x in self.X:
            x.zero_()
        arr = (_BatchItem * len(items))()
        for i, m in enumerate(self.meshes):
            arr[i] = _BatchItem(m.handle.value, self.ks[i], self.X[i].data_ptr(), m.nv, self.Y[i].data_ptr(), m.nv)
        flags = (0 if graph else 0x1) | (0x2 if autotune else 0) | (0x4 if cuda_cores else 0)
        h = ctypes.c_void_p()
        _check(load().gyps_batch_create(arr, len(items), int(nrhs), flags, _stream(stream), ctypes.byref(h)))
        self._h = h
        info = _BatchInfo()
        _check(load().gyps_batch_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _BatchInfo._fields_}
        del torch

    def apply(self, stream=None):
        _check(load().gyps_batch_apply(self._h, _stream(stream)))
        return self.Y

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            code = _lib.gyps_batch_destroy(self._h)
            self._h = None
            _check(code)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Precond:
    """Learned message-passing preconditioner (gyps_precond_*): z = M(r) ~ V^{-1} r."""

    def __init__(self, hidden: int = 64, layers: int = 4, seed: int = 995):
        h = ctypes.c_void_p()
        _check(load().gyps_precond_create(int(hidden), int(layers), int(seed), ctypes.byref(h)))
        self._h = h
        hid, lay, npar, steps = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().gyps_precond_info(self._h, ctypes.byref(hid), ctypes.byref(lay), ctypes.byref(npar),
                                        ctypes.byref(steps)))
        self.hidden, self.layers, self.nparams = hid.value, lay.value, npar.value

    @property
    def handle(self):
        return self._h

    def steps(self) -> int:
        s = ctypes.c_int64()
        _check(load().gyps_precond_info(self._h, None, None, None, ctypes.byref(s)))
        return s.value

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(load().gyps_precond_params(self._h, out.ctypes.data, self.nparams, 0))
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        _check(load().gyps_precond_params(self._h, p.ctypes.data, p.size, 1))

    def apply(self, mesh: "Mesh", k: float, R, stream=None):
        r, nrhs, ldr = _colmajor(R, mesh.nv, "R")
        z = _empty_colmajor(mesh.nv, nrhs, r.device)
        _check(load().gyps_precond_apply(self._h, mesh.handle, float(k), nrhs, r.data_ptr(), ldr, z.data_ptr(),
                                         mesh.nv, _stream(stream)))
        return z

    def train_step(self, mesh: "Mesh", k: float, R, E, lr: float, want_grad: bool = False, stream=None):
        """Loss (and gradient) on the minibatch; one Adam step when lr > 0."""
        r, nrhs, ldr = _colmajor(R, mesh.nv, "R")
        e, nrhs_e, lde = _colmajor(E, mesh.nv, "E")
        if nrhs_e != nrhs:
            raise ValueError("R and E must have the same number of columns")
        loss = ctypes.c_double()
        grad = np.zeros(self.nparams, dtype=np.float32) if want_grad else None
        _check(load().gyps_precond_train_step(self._h, mesh.handle, float(k), nrhs, r.data_ptr(), ldr, e.data_ptr(),
                                              lde, float(lr), ctypes.byref(loss),
                                              grad.ctypes.data if grad is not None else None, _stream(stream)))
        return (loss.value, grad) if want_grad else loss.value

    def range(self):
        """(ka_lo, ka_hi): electrical sizes k x radius trained on (lo > hi: none)."""
        lo, hi = ctypes.c_double(), ctypes.c_double()
        _check(load().gyps_precond_range(self.handle, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def save(self, path: str) -> None:
        _check(load().gyps_precond_save(self._h, str(path).encode()))

    def load(self, path: str) -> None:
        _check(load().gyps_precond_load(self._h, str(path).encode()))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.gyps_precond_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class GmresReport:
    iterations: int
    applies: int
    check_applies: int
    refinements: int
    precond_fallback: int
    est_residual: np.ndarray
    true_residual: np.ndarray
    converged: np.ndarray
    status: str


FORMULATION = {"sl": 0, "bw": 1, "cfie": 2, "efie": 3, "emcfie": 4}


def gmres_solve(mesh: Mesh, k: float, F, tol: float = 1e-6, restart: int = 100, maxit: int = 1000,
                prec: str = "fp32", check_prec: str = "fp64", x0=None, max_refine: int = 3, raise_on_fail=False,
                precond: "Precond" = None, stream=None, formulation: str = "sl", eta: float = None,
                timeout_ms: float = 0.0, hmat: "Hmat" = None):
    """Solves A X = F (gyps_gmres_solve), A = V ("sl"), 1/2 M + K - i eta V ("bw"),
    1/2 M + K' - i eta V ("cfie"; F from rhs_planewave_cfie with the same eta) or -T
    ("efie"; RWG coefficients, F from rhs_planewave_efie), or -eta T + (1 - eta)(Id/2 - nxK)
    ("emcfie", eta = beta; F from rhs_planewave_emcfie); eta defaults to k, or 1 at
    k = 0.  timeout_ms > 0 bounds the wall-clock time (status TIMEOUT, X = last iterate).
    prec="hmat" takes the compressed operator `hmat` (built for this mesh and k) in the
    Krylov loop; check_prec then judges the residual with a kernel product.
    Returns (X, GmresReport); NOT_CONVERGED and TIMEOUT raise only with raise_on_fail."""
    if eta is None:
        eta = 0.5 if formulation == "emcfie" else (float(k) if k > 0 else 1.0)
    n = rwg_edges(mesh, stream)[0] if formulation in ("efie", "emcfie") else mesh.nv
    f, nrhs, ldf = _colmajor(F, n, "F")
    if x0 is not None:
        x, _, _ = _colmajor(x0.clone() if hasattr(x0, "clone") else x0, n, "x0")
        x = x.to(f.device)
        if x.stride(1) != n and nrhs > 1:
            x = x.t().contiguous().t()
    else:
        x = _empty_colmajor(n, nrhs, f.device)
    opts = _GmresOpts(float(tol), int(restart), int(maxit), PREC[prec], PREC[check_prec], 1 if x0 is not None else 0,
                      int(max_refine), precond.handle.value if precond is not None else None,
                      FORMULATION[formulation], float(eta), float(timeout_ms),
                      hmat._h.value if hmat is not None else None)
    est = np.zeros(nrhs)
    tru = np.zeros(nrhs)
    conv = np.zeros(nrhs, dtype=np.int32)
    rep = _GmresReport(0, 0, 0, 0, 0, est.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       tru.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       conv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    code = load().gyps_gmres_solve(mesh.handle, float(k), nrhs, f.data_ptr(), ldf, x.data_ptr(), n,
                                   ctypes.byref(opts), ctypes.byref(rep), _stream(stream))
    wall_clock = False
    if code == 6:  # TIMEOUT: GMRES's own wall-clock limit, or a device wait that ran out (always raised)
        buf = ctypes.create_string_buffer(512)
        load().gyps_last_error(buf, 512)
        wall_clock = b"wall-clock" in buf.value
    if code not in (0, 4, 6) or (code == 6 and not wall_clock) or (code in (4, 6) and raise_on_fail):
        _check(code)
    report = GmresReport(rep.iterations, rep.applies, rep.check_applies, rep.refinements, rep.precond_fallback, est,
                         tru, conv.astype(bool), _STATUS[code])
    return (x[:, 0] if (hasattr(F, "dim") and F.dim() == 1) else x), report
