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
        ("eps_field", C.POINTER(C.c_double)), ("K_field", C.POINTER(C.c_double)),
        ("round_nearest", C.c_int),
    ]


class lbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("eps", C.c_double), ("sigma", C.c_double),
        ("varpi", C.c_double), ("nu", C.c_double), ("K", C.c_double), ("Feps", C.c_double),
        ("gbT", C.c_double), ("gbC", C.c_double), ("Gx", C.c_double), ("T0", C.c_double),
        ("C0", C.c_double), ("s", C.c_double * 9), ("zeta", C.c_double * 5),
        ("eta", C.c_double * 5), ("Tw", C.c_double * 4), ("Cw", C.c_double * 4),
        ("wall_lr", C.c_int), ("wall_tb", C.c_int), ("uw", (C.c_double * 2) * 4),
        ("model_a", C.c_int), ("nee", C.c_int), ("BiT", C.c_double * 4), ("BiC", C.c_double * 4),
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
            L.lbm_params_model_a.argtypes = [C.POINTER(lbm_params)]
            L.lbm_derive_params_lid.argtypes = [lbm_grid] + [C.c_double] * 11 + [C.POINTER(lbm_params)]
            L.lbm_derive_params_nee.argtypes = [lbm_grid] + [C.c_double] * 10 + [C.POINTER(lbm_params)]
            L.lbm_derive_params_lid_nee.argtypes = [lbm_grid] + [C.c_double] * 11 + [C.POINTER(lbm_params)]
            L.lbm_derive_params_convective.argtypes = ([C.c_int] + [C.c_double] * 12
                                                       + [C.POINTER(lbm_params)])
            L.lbm_nusselt_sherwood_tb.argtypes = [P, dp]
            L.lbm_reset.argtypes = [P, dp, dp, C.c_uint64, C.c_double]
            L.lbm_step.argtypes = [P, C.c_int64]
            L.lbm_time.argtypes = [P]
            L.lbm_time.restype = C.c_int64
            L.lbm_fields.argtypes = [P, dp, dp, dp, dp, dp]
            L.lbm_fields_window.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.lbm_nusselt_sherwood.argtypes = [P, dp]
            L.lbm_residual.argtypes = [P, dp]
            L.lbm_residual_noalloc.argtypes = [P, C.c_void_p, C.c_int, dp]
            L.lbm_residual_parts.argtypes = [P, dp]
            L.lbm_create_slab.argtypes = [C.POINTER(lbm_params), C.c_int, C.c_int,
                                          C.POINTER(lbm_options), C.POINTER(C.c_void_p)]
            L.lbm_halo_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
            L.lbm_halo_export.argtypes = [P, C.c_int, C.c_void_p]
            L.lbm_halo_import.argtypes = [P, C.c_int, C.c_void_p]
            L.lbm_save.argtypes = [P, C.c_void_p, C.POINTER(C.c_size_t)]
            L.lbm_load.argtypes = [P, C.c_void_p, C.c_size_t]
            L.lbm_get_params.argtypes = [P, C.POINTER(lbm_params)]
            L.lbm_device_bytes.argtypes = [P]
            L.lbm_device_bytes.restype = C.c_size_t
            L.lbm_destroy.argtypes = [P]
            L.lbm_last_error.argtypes = [P]
            L.lbm_last_error.restype = C.c_char_p
            for name in ("lbm_derive_params", "lbm_params_model_a", "lbm_derive_params_lid",
                         "lbm_derive_params_nee", "lbm_derive_params_convective",
                         "lbm_derive_params_lid_nee",
                         "lbm_nusselt_sherwood_tb", "lbm_create", "lbm_create_raw",
                         "lbm_reset", "lbm_step",
                         "lbm_fields", "lbm_fields_window", "lbm_nusselt_sherwood", "lbm_residual",
                         "lbm_residual_noalloc", "lbm_residual_parts", "lbm_create_slab",
                         "lbm_halo_bytes", "lbm_halo_export", "lbm_halo_import", "lbm_save",
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


def lbm_derive_params_lid(nx, ny, Re, Gr, Da, eps, Pr, Le, N, J=1.0, sigma=1.0, U0=0.1,
                          varpi=0.0):
    p = lbm_params()
    _check(lib().lbm_derive_params_lid(lbm_grid(int(nx), int(ny)), Re, Gr, Da, eps, Pr, Le, N, J,
                                       sigma, U0, varpi, C.byref(p)))
    return p


def lbm_derive_params_nee(nx, ny, Ra, Da, eps, Pr, Le, N, J=1.0, sigma=1.0, Ma=0.0, varpi=0.0):
    """lbm_derive_params for walls with nodes on them (Sec. 3.3), L = nx - 1."""
    p = lbm_params()
    _check(lib().lbm_derive_params_nee(lbm_grid(int(nx), int(ny)), Ra, Da, eps, Pr, Le, N, J, sigma,
                                       Ma, varpi, C.byref(p)))
    return p


def lbm_derive_params_convective(Nx, Ra, Da, eps, Pr, Le, N, BiT, BiC, J=1.0, sigma=1.0, Ma=0.0,
                                 varpi=0.0):
    """The porous cavity with a freely convective right wall of Sec. 4.2 (Nx spacings,
    Nx + 1 nodes per side on the walls)."""
    p = lbm_params()
    _check(lib().lbm_derive_params_convective(int(Nx), Ra, Da, eps, Pr, Le, N, BiT, BiC, J, sigma,
                                              Ma, varpi, C.byref(p)))
    return p


def lbm_derive_params_lid_nee(nx, ny, Re, Gr, Da, eps, Pr, Le, N, J=1.0, sigma=1.0, U0=0.1,
                              varpi=0.0):
    """lbm_derive_params_lid for walls with nodes on them (Sec. 3.3), L = nx - 1."""
    p = lbm_params()
    _check(lib().lbm_derive_params_lid_nee(lbm_grid(int(nx), int(ny)), Re, Gr, Da, eps, Pr, Le, N,
                                           J, sigma, U0, varpi, C.byref(p)))
    return p


def lbm_params_model_a(p: lbm_params) -> lbm_params:
    _check(lib().lbm_params_model_a(C.byref(p)))
    return p


class Cavity:
    """One cavity on the device (wraps an lbm_ctx*)."""

    def __init__(self, nx=None, ny=None, Ra=None, Da=None, eps=None, Pr=1.0, Le=1.0, N=1.0,
                 J=1.0, sigma=1.0, *, params: lbm_params | None = None, precision="f64",
                 layout="ab", Ma=0.0, varpi=0.0, seed=1, noise=1e-3, T_init=None, C_init=None,
                 stream=None, allocator="torch", block=(0, 0), graph_chunk=0,
                 round_nearest=False, eps_field=None, K_field=None, slab=None):
        """slab=(y0, h): the rows [y0, y0 + h) of the cavity given by `params`
        (lbm_create_slab); exchange faces with halo_export / halo_import."""
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
        o.round_nearest = int(bool(round_nearest))
        for name, arr in (("eps_field", eps_field), ("K_field", K_field)):
            if arr is not None:
                a = np.ascontiguousarray(arr, dtype=np.float64)
                self._keep.append(a)
                setattr(o, name, _dptr(a))
        h = C.c_void_p()
        if slab is not None:
            st = L.lbm_create_slab(C.byref(params), int(slab[0]), int(slab[1]), C.byref(o),
                                   C.byref(h))
        elif params is not None:
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
        if slab is not None:
            self.y0, self.ny = int(slab[0]), int(slab[1])

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

    def fields_window(self, x0, y0, w, h, which=("ux", "uy", "T", "C", "rho")):
        out = {k: np.empty((h, w)) for k in which}
        args = [_dptr(out.get(k)) for k in ("ux", "uy", "T", "C", "rho")]
        _check(lib().lbm_fields_window(self.h, int(x0), int(y0), int(w), int(h), *args), self.h)
        return out

    def nusselt_sherwood(self):
        out = np.empty(4)
        _check(lib().lbm_nusselt_sherwood(self.h, _dptr(out)), self.h)
        return out

    def nusselt_sherwood_tb(self):
        out = np.empty(4)
        _check(lib().lbm_nusselt_sherwood_tb(self.h, _dptr(out)), self.h)
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

    def residual_parts(self) -> np.ndarray:
        """lbm_residual_parts: max |phi - phi_snap| (4) and max |phi| (4) of u_x, u_y, T, C."""
        out = np.empty(8)
        _check(lib().lbm_residual_parts(self.h, _dptr(out)), self.h)
        return out

    def halo_bytes(self) -> int:
        n = C.c_size_t()
        _check(lib().lbm_halo_bytes(self.h, C.byref(n)), self.h)
        return n.value

    def halo_export(self, side: int, face_ptr: int):
        _check(lib().lbm_halo_export(self.h, int(side), C.c_void_p(int(face_ptr))), self.h)

    def halo_import(self, side: int, face_ptr: int):
        _check(lib().lbm_halo_import(self.h, int(side), C.c_void_p(int(face_ptr))), self.h)

    def save(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib().lbm_save(self.h, None, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(lib().lbm_save(self.h, buf, C.byref(n)), self.h)
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().lbm_load(self.h, buf, len(blob)), self.h)
        p = lbm_params()                      # the checkpoint brings its own parameters
        _check(lib().lbm_get_params(self.h, C.byref(p)), self.h)
        self.params = p

    def device_bytes(self) -> int:
        return int(lib().lbm_device_bytes(self.h))


class lbm_instance(C.Structure):
    _fields_ = [("params", lbm_params), ("seed", C.c_uint64), ("noise", C.c_double)]


_batch_ready = False


def _batch_lib():
    global _batch_ready
    L = lib()
    if not _batch_ready:
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.lbm_batch_create.argtypes = [C.POINTER(lbm_instance), C.c_int, C.c_int, C.c_size_t,
                                       C.POINTER(lbm_options), C.POINTER(C.c_void_p)]
        L.lbm_batch_instance_bytes.argtypes = [lbm_grid, C.POINTER(lbm_options)]
        L.lbm_batch_instance_bytes.restype = C.c_size_t
        L.lbm_batch_add.argtypes = [P, C.POINTER(lbm_instance), C.POINTER(C.c_int)]
        L.lbm_batch_remove.argtypes = [P, C.c_int]
        L.lbm_batch_step.argtypes = [P, C.c_int64]
        L.lbm_batch_time.argtypes = [P, C.c_int]
        L.lbm_batch_time.restype = C.c_int64
        L.lbm_batch_nusselt_sherwood.argtypes = [P, dp]
        L.lbm_batch_residual.argtypes = [P, dp, C.POINTER(C.c_int)]
        L.lbm_batch_fields.argtypes = [P, C.c_int, dp, dp, dp, dp, dp]
        L.lbm_batch_autotune.argtypes = [P, C.c_int, C.c_char_p, C.c_size_t]
        L.lbm_batch_set_tile.argtypes = [P, C.c_int, C.c_int, C.c_int]
        L.lbm_batch_set_blocking.argtypes = [P, C.c_int, C.c_size_t]
        L.lbm_batch_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        L.lbm_batch_destroy.argtypes = [P]
        L.lbm_batch_last_error.argtypes = [P]
        L.lbm_batch_last_error.restype = C.c_char_p
        for n in ("lbm_batch_create", "lbm_batch_add", "lbm_batch_remove", "lbm_batch_step",
                  "lbm_batch_nusselt_sherwood", "lbm_batch_residual", "lbm_batch_fields",
                  "lbm_batch_autotune", "lbm_batch_info", "lbm_batch_set_tile",
                  "lbm_batch_set_blocking"):
            getattr(L, n).restype = C.c_int
        _batch_ready = True
    return L


def _bcheck(status, handle=None):
    if status != OK:
        msg = _batch_lib().lbm_batch_last_error(handle).decode(errors="replace")
        raise LbmError(status, msg)


def make_instance(spec=None, *, params=None, seed=1, noise=1e-3) -> lbm_instance:
    """Instance descriptor from a workloads.CavitySpec (or explicit lbm_params)."""
    inst = lbm_instance()
    if params is None:
        params = lbm_derive_params(*spec.args(), varpi=getattr(spec, "varpi", 0.0))
        seed, noise = spec.seed, spec.noise
    inst.params = params
    inst.seed = int(seed)
    inst.noise = -1.0 if noise == 0 else float(noise)
    return inst


def _options(precision, layout, stream, allocator, graph_chunk, round_nearest):
    o = lbm_options()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    if stream is not None:
        o.stream = int(stream)
    keep = None
    if allocator == "torch":
        keep = TorchAllocator()
        o.alloc, o.free = keep.alloc, keep.free
    o.graph_chunk = int(graph_chunk)
    o.round_nearest = int(bool(round_nearest))
    return o, keep


def batch_instance_bytes(nx, ny, precision="f32", layout="ab") -> int:
    o, _ = _options(precision, layout, None, None, 0, False)
    return int(_batch_lib().lbm_batch_instance_bytes(lbm_grid(int(nx), int(ny)), C.byref(o)))


class Batch:
    """Many cavities advanced by one fused launch per step (wraps lbm_batch*)."""

    def __init__(self, instances=(), capacity=None, arena_bytes=0, *, precision="f32", layout="ab",
                 stream=None, allocator="torch", graph_chunk=0, round_nearest=False):
        L = _batch_lib()
        insts = list(instances)
        cap = int(capacity if capacity is not None else max(1, len(insts)))
        o, self._alloc = _options(precision, layout, stream, allocator, graph_chunk, round_nearest)
        arr = (lbm_instance * max(1, len(insts)))(*insts) if insts else None
        h = C.c_void_p()
        _bcheck(L.lbm_batch_create(arr, len(insts), cap, int(arena_bytes), C.byref(o), C.byref(h)))
        self.h = h
        self.capacity = cap
        self.shapes = {}
        for k, inst in enumerate(insts):
            self.shapes[k] = (inst.params.ny, inst.params.nx)

    def close(self):
        if getattr(self, "h", None):
            _batch_lib().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def add(self, inst: lbm_instance) -> int:
        slot = C.c_int(-1)
        _bcheck(_batch_lib().lbm_batch_add(self.h, C.byref(inst), C.byref(slot)), self.h)
        self.shapes[slot.value] = (inst.params.ny, inst.params.nx)
        return slot.value

    def remove(self, slot: int):
        _bcheck(_batch_lib().lbm_batch_remove(self.h, int(slot)), self.h)
        self.shapes.pop(slot, None)

    def step(self, n=1):
        _bcheck(_batch_lib().lbm_batch_step(self.h, int(n)), self.h)

    def time(self, slot) -> int:
        return int(_batch_lib().lbm_batch_time(self.h, int(slot)))

    def nusselt_sherwood(self) -> np.ndarray:
        out = np.zeros(4 * self.capacity)
        _bcheck(_batch_lib().lbm_batch_nusselt_sherwood(self.h, _dptr(out)), self.h)
        return out.reshape(self.capacity, 4)

    def residual(self):
        r = np.zeros(self.capacity)
        d = (C.c_int * self.capacity)()
        _bcheck(_batch_lib().lbm_batch_residual(self.h, _dptr(r), d), self.h)
        return r, np.array(d[:], dtype=bool)

    def fields(self, slot, which=("ux", "uy", "T", "C", "rho")):
        shp = self.shapes[slot]
        out = {k: np.empty(shp) for k in which}
        args = [_dptr(out.get(k)) for k in ("ux", "uy", "T", "C", "rho")]
        _bcheck(_batch_lib().lbm_batch_fields(self.h, int(slot), *args), self.h)
        return out

    def autotune(self, trial_steps=20) -> str:
        buf = C.create_string_buffer(8192)
        _bcheck(_batch_lib().lbm_batch_autotune(self.h, int(trial_steps), buf, 8192), self.h)
        return buf.value.decode()

    def set_tile(self, slot, tile_w, tile_h):
        _bcheck(_batch_lib().lbm_batch_set_tile(self.h, int(slot), int(tile_w), int(tile_h)),
                self.h)

    def set_blocking(self, steps, l2_bytes=0):
        _bcheck(_batch_lib().lbm_batch_set_blocking(self.h, int(steps), int(l2_bytes)), self.h)

    def info(self):
        cap, used = C.c_int(), C.c_int()
        ab, au = C.c_size_t(), C.c_size_t()
        _bcheck(_batch_lib().lbm_batch_info(self.h, C.byref(cap), C.byref(used), C.byref(ab),
                                            C.byref(au)), self.h)
        return {"capacity": cap.value, "used": used.value, "arena_bytes": ab.value,
                "arena_used": au.value}


class lbm_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("steps", C.c_int64),
                ("residual", C.c_double), ("nush", C.c_double * 4), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


_server_ready = False


def _server_lib():
    global _server_ready
    L = _batch_lib()
    if not _server_ready:
        P = C.c_void_p
        L.lbm_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.POINTER(lbm_options),
                                        C.POINTER(C.c_void_p)]
        L.lbm_server_submit.argtypes = [P, C.POINTER(lbm_instance), C.c_double, C.c_double,
                                        C.c_int64, C.c_int64]
        L.lbm_server_tick.argtypes = [P, C.POINTER(C.c_int)]
        L.lbm_server_poll.argtypes = [P, C.POINTER(lbm_result), C.c_int, C.POINTER(C.c_int)]
        L.lbm_server_clock.argtypes = [P]
        L.lbm_server_clock.restype = C.c_double
        L.lbm_server_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
        L.lbm_server_destroy.argtypes = [P]
        L.lbm_server_last_error.argtypes = [P]
        L.lbm_server_last_error.restype = C.c_char_p
        for n in ("lbm_server_create", "lbm_server_submit", "lbm_server_tick", "lbm_server_poll",
                  "lbm_server_info"):
            getattr(L, n).restype = C.c_int
        _server_ready = True
    return L


def _scheck(status, handle=None):
    if status != OK:
        msg = _server_lib().lbm_server_last_error(handle).decode(errors="replace")
        raise LbmError(status, msg)


class Server:
    """Continuous-batching solver service (wraps lbm_server*)."""

    def __init__(self, budget_bytes, max_slots=256, check_every=100, *, precision="bf16",
                 layout="ab", stream=None, allocator="torch", graph_chunk=0, round_nearest=False):
        L = _server_lib()
        o, self._alloc = _options(precision, layout, stream, allocator, graph_chunk, round_nearest)
        h = C.c_void_p()
        _scheck(L.lbm_server_create(int(budget_bytes), int(max_slots), int(check_every),
                                    C.byref(o), C.byref(h)))
        self.h = h
        self._buf = (lbm_result * 1024)()

    def close(self):
        if getattr(self, "h", None):
            _server_lib().lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def submit(self, inst: lbm_instance, tol=1e-7, max_steps=10 ** 7, rid=0, nush_tol=0.0):
        _scheck(_server_lib().lbm_server_submit(self.h, C.byref(inst), float(tol), float(nush_tol),
                                                int(max_steps), int(rid)), self.h)

    def tick(self) -> int:
        n = C.c_int(0)
        _scheck(_server_lib().lbm_server_tick(self.h, C.byref(n)), self.h)
        return n.value

    def poll(self):
        out = []
        while True:
            n = C.c_int(0)
            _scheck(_server_lib().lbm_server_poll(self.h, self._buf, 1024, C.byref(n)), self.h)
            for k in range(n.value):
                r = self._buf[k]
                out.append({"id": r.id, "status": r.status, "steps": r.steps,
                            "residual": r.residual, "nush": list(r.nush), "t_submit": r.t_submit,
                            "t_admit": r.t_admit, "t_done": r.t_done})
            if n.value < 1024:
                return out

    def clock(self) -> float:
        return float(_server_lib().lbm_server_clock(self.h))

    def info(self):
        q, a, d = C.c_int(), C.c_int(), C.c_int()
        m = C.c_size_t()
        _scheck(_server_lib().lbm_server_info(self.h, C.byref(q), C.byref(a), C.byref(d),
                                              C.byref(m)), self.h)
        return {"queued": q.value, "active": a.value, "done": d.value, "arena_used": m.value}

    def drain(self, max_ticks=10 ** 7):
        """Tick until queue and slots are empty; returns all results."""
        res = []
        for _ in range(max_ticks):
            active = self.tick()
            res += self.poll()
            inf = self.info()
            if active == 0 and inf["queued"] == 0:
                break
        return res + self.poll()
