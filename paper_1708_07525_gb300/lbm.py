"""Thin ctypes binding of liblbm (include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of liblbm.so.  PyTorch supplies device memory (its caching allocator, through
the allocator hooks of lbm_options) and the CUDA stream.  If the shared
library cannot be loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

F64, F32, BF16, F16 = 0, 1, 2, 3
AB_PULL, AA = 0, 1
WALL_DIRICHLET, WALL_ADIABATIC = 0, 1
PRECISIONS = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}
LAYOUTS = {"ab": AB_PULL, "aa": AA}
NOALLOC_MAX_NODES = 4096 * 1024   # LBM_NOALLOC_MAX_NODES

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_UNCONVERGED = range(7)
_STATUS = {1: "LBM_ERR_INVALID", 2: "LBM_ERR_NOMEM", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_DIVERGED",
           5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_UNCONVERGED"}


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class lbm_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("layout", C.c_int), ("Ma", C.c_double), ("varpi", C.c_double),
        ("seed", C.c_uint64), ("noise", C.c_double),
        ("T_init", C.POINTER(C.c_double)), ("C_init", C.POINTER(C.c_double)),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
        ("block_x", C.c_int), ("block_y", C.c_int), ("graph_chunk", C.c_int),
    ]


class lbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("eps", C.c_double), ("sigma", C.c_double),
        ("varpi", C.c_double), ("nu", C.c_double), ("K", C.c_double), ("Feps", C.c_double),
        ("gbT", C.c_double), ("gbC", C.c_double), ("Gx", C.c_double), ("T0", C.c_double),
        ("C0", C.c_double), ("s", C.c_double * 9), ("zeta", C.c_double * 5),
        ("eta", C.c_double * 5), ("Tw", C.c_double * 4), ("Cw", C.c_double * 4),
        ("wall_lr", C.c_int), ("wall_tb", C.c_int),
    ]


_lib = None
_lock = threading.Lock()


def lib():
    """Load liblbm.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            L = C.CDLL(path)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.lbm_derive_params.argtypes = [lbm_grid] + [C.c_double] * 10 + [C.POINTER(lbm_params)]
            L.lbm_create.argtypes = [lbm_grid] + [C.c_double] * 8 + [C.POINTER(lbm_options),
                                                                     C.POINTER(C.c_void_p)]
            L.lbm_create_raw.argtypes = [C.POINTER(lbm_params), C.POINTER(lbm_options),
                                         C.POINTER(C.c_void_p)]
            L.lbm_reset.argtypes = [P, dp, dp, C.c_uint64, C.c_double]
            L.lbm_step.argtypes = [P, C.c_int64]
            L.lbm_time.argtypes = [P]
            L.lbm_time.restype = C.c_int64
            L.lbm_fields.argtypes = [P, dp, dp, dp, dp, dp]
            L.lbm_nusselt_sherwood.argtypes = [P, dp]
            L.lbm_residual.argtypes = [P, dp]
            L.lbm_residual_noalloc.argtypes = [P, C.c_void_p, C.c_int, dp]
            L.lbm_save.argtypes = [P, C.c_void_p, C.POINTER(C.c_size_t)]
            L.lbm_load.argtypes = [P, C.c_void_p, C.c_size_t]
            L.lbm_get_params.argtypes = [P, C.POINTER(lbm_params)]
            L.lbm_device_bytes.argtypes = [P]
            L.lbm_device_bytes.restype = C.c_size_t
            L.lbm_destroy.argtypes = [P]
            L.lbm_last_error.argtypes = [P]
            L.lbm_last_error.restype = C.c_char_p
            for name in ("lbm_derive_params", "lbm_create", "lbm_create_raw", "lbm_reset", "lbm_step",
                         "lbm_fields", "lbm_nusselt_sherwood", "lbm_residual",
                         "lbm_residual_noalloc", "lbm_save",
                         "lbm_load", "lbm_get_params"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(status, handle=None):
    if status != OK:
        msg = lib().lbm_last_error(handle).decode(errors="replace")
        raise LbmError(status, msg)


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


class TorchAllocator:
    """Allocator hooks backed by PyTorch's CUDA caching allocator."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device

        def _alloc(nbytes, user, stream):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              int(stream or 0)))
            except Exception:  # out of memory -> NULL, reported as LBM_ERR_NOMEM
                return None

        def _free(ptr, user, stream):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def torch_stream_handle(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def lbm_derive_params(nx, ny, Ra, Da, eps, Pr, Le, N, J=1.0, sigma=1.0, Ma=0.0, varpi=0.0):
    p = lbm_params()
    _check(lib().lbm_derive_params(lbm_grid(int(nx), int(ny)), Ra, Da, eps, Pr, Le, N, J, sigma,
                                   Ma, varpi, C.byref(p)))
    return p


class Cavity:
    """One cavity on the device (wraps an lbm_ctx*)."""

    def __init__(self, nx=None, ny=None, Ra=None, Da=None, eps=None, Pr=1.0, Le=1.0, N=1.0,
                 J=1.0, sigma=1.0, *, params: lbm_params | None = None, precision="f64",
                 layout="ab", Ma=0.0, varpi=0.0, seed=1, noise=1e-3, T_init=None, C_init=None,
                 stream=None, allocator="torch", block=(0, 0), graph_chunk=0):
        L = lib()
        o = lbm_options()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        o.Ma, o.varpi, o.seed = Ma, varpi, int(seed)
        o.noise = -1.0 if noise == 0 else float(noise)
        self._keep = []
        if T_init is not None:
            Ti = np.ascontiguousarray(T_init, dtype=np.float64)
            Ci = np.ascontiguousarray(C_init, dtype=np.float64)
            self._keep += [Ti, Ci]
            o.T_init, o.C_init = _dptr(Ti), _dptr(Ci)
        if stream is not None:
            o.stream = int(stream)
        if allocator == "torch":
            self._alloc = TorchAllocator()
            o.alloc, o.free = self._alloc.alloc, self._alloc.free
        o.block_x, o.block_y = int(block[0]), int(block[1])
        o.graph_chunk = int(graph_chunk)
        h = C.c_void_p()
        if params is not None:
            st = L.lbm_create_raw(C.byref(params), C.byref(o), C.byref(h))
        else:
            st = L.lbm_create(lbm_grid(int(nx), int(ny)), Ra, Da, eps, Pr, Le, N, J, sigma,
                              C.byref(o), C.byref(h))
        _check(st)
        self.h = h
        p = lbm_params()
        _check(L.lbm_get_params(self.h, C.byref(p)), self.h)
        self.params = p
        self.nx, self.ny = p.nx, p.ny

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def t(self) -> int:
        return int(lib().lbm_time(self.h))

    def reset(self, T_init=None, C_init=None, seed=1, noise=1e-3, T_ptr=None, C_ptr=None):
        """Back to t = 0 from host fields (numpy arrays, or raw host pointers T_ptr /
        C_ptr, e.g. of pinned torch tensors) or from the seeded noise."""
        dp = C.POINTER(C.c_double)
        if T_ptr is not None:
            Tp, Cp = C.cast(C.c_void_p(T_ptr), dp), C.cast(C.c_void_p(C_ptr), dp)
        elif T_init is not None:
            self._reset_keep = (np.ascontiguousarray(T_init, dtype=np.float64),
                                np.ascontiguousarray(C_init, dtype=np.float64))
            Tp, Cp = (_dptr(a) for a in self._reset_keep)
        else:
            Tp = Cp = None
        _check(lib().lbm_reset(self.h, Tp, Cp, int(seed), -1.0 if noise == 0 else float(noise)),
               self.h)

    def step(self, n=1):
        _check(lib().lbm_step(self.h, int(n)), self.h)

    def fields(self, which=("ux", "uy", "T", "C", "rho")):
        shp = (self.ny, self.nx)
        out = {k: np.empty(shp) for k in which}
        args = [_dptr(out.get(k)) for k in ("ux", "uy", "T", "C", "rho")]
        _check(lib().lbm_fields(self.h, *args), self.h)
        return out

    def nusselt_sherwood(self):
        out = np.empty(4)
        _check(lib().lbm_nusselt_sherwood(self.h, _dptr(out)), self.h)
        return out

    def residual(self):
        r = C.c_double()
        _check(lib().lbm_residual(self.h, C.byref(r)), self.h)
        return r.value

    def residual_noalloc(self, snapshot_ptr: int, have_snapshot: bool) -> float:
        """lbm_residual_noalloc: residual against a caller-owned device snapshot of
        4 * nx * ny doubles; the library allocates nothing for this call."""
        r = C.c_double()
        _check(lib().lbm_residual_noalloc(self.h, C.c_void_p(int(snapshot_ptr)),
                                          int(bool(have_snapshot)), C.byref(r)), self.h)
        return r.value

    def save(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib().lbm_save(self.h, None, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(lib().lbm_save(self.h, buf, C.byref(n)), self.h)
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().lbm_load(self.h, buf, len(blob)), self.h)

    def device_bytes(self) -> int:
        return int(lib().lbm_device_bytes(self.h))
