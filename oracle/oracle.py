"""ctypes wrapper around the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline / reference leg.  The GPU library never imports it.

The oracle follows the paper section by section (Liu & He, arXiv:1708.07525):
Sec. 3.1 (Eqs. 8-20) for the flow lattice, Sec. 3.2 (Eqs. 21-28) for the
temperature and concentration lattices, Eq. 11 for streaming and Eq. 38 for
the Nusselt / Sherwood numbers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "lbm_oracle.c")]
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_lock = threading.Lock()
_lib = None

DIRICHLET = 0
ADIABATIC = 1


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("Ra", C.c_double), ("Da", C.c_double), ("eps", C.c_double), ("Pr", C.c_double),
        ("Le", C.c_double), ("N", C.c_double), ("J", C.c_double), ("sigma", C.c_double),
        ("Ma", C.c_double), ("varpi", C.c_double),
        ("rho0", C.c_double), ("cs2", C.c_double), ("U", C.c_double), ("nu", C.c_double),
        ("nu_e", C.c_double), ("alpha_e", C.c_double), ("D_e", C.c_double),
        ("csT2", C.c_double), ("K", C.c_double), ("Feps", C.c_double), ("gbT", C.c_double),
        ("gbC", C.c_double), ("T0", C.c_double), ("C0", C.c_double),
        ("s", C.c_double * 9), ("zeta", C.c_double * 5), ("eta", C.c_double * 5),
        ("periodic_x", C.c_int), ("periodic_y", C.c_int),
        ("scalar_lr", C.c_int), ("scalar_tb", C.c_int),
        ("Tw", C.c_double * 4), ("Cw", C.c_double * 4),
        ("uw", (C.c_double * 2) * 4),
        ("Gx", C.c_double),
        ("model_a", C.c_int),
        ("nee", C.c_int),
        ("BiT", C.c_double * 4), ("BiC", C.c_double * 4),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so with gcc (plain -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # LBM_ORACLE_LIB names another compiled copy of the oracle to load instead
            # (the planted-mistake test builds altered copies and runs the pins on them)
            L = C.CDLL(os.environ.get("LBM_ORACLE_LIB") or build())
            P = C.POINTER(Params)
            dp = C.POINTER(C.c_double)
            L.or_derive.argtypes = [P]
            L.or_derive.restype = C.c_int
            L.or_create.argtypes = [P, C.c_uint64, C.c_double, dp, dp]
            L.or_create.restype = C.c_void_p
            L.or_create_field.argtypes = [P, C.c_uint64, C.c_double, dp, dp, dp, dp]
            L.or_create_field.restype = C.c_void_p
            L.or_destroy.argtypes = [C.c_void_p]
            L.or_step.argtypes = [C.c_void_p, C.c_long]
            L.or_time.argtypes = [C.c_void_p]
            L.or_time.restype = C.c_long
            L.or_fields.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            L.or_nusselt_sherwood.argtypes = [C.c_void_p, dp]
            L.or_nusselt_sherwood_tb.argtypes = [C.c_void_p, dp]
            L.or_stream_function.argtypes = [C.c_void_p, dp]
            L.or_residual_fields.argtypes = [C.c_long, dp, dp, dp]
            L.or_residual_fields.restype = C.c_int
            L.or_residual.argtypes = [C.c_void_p, dp, C.c_int, dp]
            L.or_residual.restype = C.c_int
            L.or_get.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.or_set.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.or_collide_node.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
            L.or_uniform.argtypes = [C.c_uint64, C.c_uint64]
            L.or_uniform.restype = C.c_double
            L.or_set_threads.argtypes = [C.c_int]
            L.or_noise_window.argtypes = [C.c_uint64, C.c_double, C.c_int, C.c_int, C.c_int,
                                          C.c_int, C.c_int, C.c_int, dp, dp]
            L.or_get_threads.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def derive(nx, ny, Ra, Da, eps, Pr, Le, N, J=1.0, sigma=1.0, Ma=0.1, varpi=0.4,
           nee=False) -> Params:
    """Parameter mapping of Sec. 4 / 4.1 (see or_derive); nee: nodes on the walls
    with the non-equilibrium extrapolation of Sec. 3.3 (then L = nx - 1)."""
    p = Params()
    p.nx, p.ny = int(nx), int(ny)
    p.nee = 1 if nee else 0
    p.Ra, p.Da, p.eps, p.Pr, p.Le, p.N, p.J, p.sigma = Ra, Da, eps, Pr, Le, N, J, sigma
    p.Ma, p.varpi = Ma, varpi
    rc = lib().or_derive(C.byref(p))
    if rc != 0:
        raise ValueError(f"invalid parameters (or_derive returned {rc})")
    return p


def derive_lid(nx, ny, Re, Gr, Da, eps, Pr, Le, N, J=1.0, sigma=1.0, U0=0.1, varpi=0.4,
               nee=False) -> Params:
    """Lid-driven porous cavity of Sec. 4.3: the top wall moves with U0 along +x, top
    T = C = 1, bottom T = C = 0, left/right adiabatic; Re = L U0 / nu with
    1/s_nu = 1/2 + J L U0 / (c_s^2 Re); Gr = g beta_T dT L^3 / nu^2 (L = nx, or nx - 1
    with nodes on the walls)."""
    p = derive(nx, ny, 1e4, Da, eps, Pr, Le, N, J, sigma, 0.1, varpi, nee=nee)
    L = float(nx - 1) if nee else float(nx)
    nu_e = J * L * U0 / Re
    p.nu_e, p.nu = nu_e, nu_e / J
    p.alpha_e = p.nu / Pr
    p.D_e = p.alpha_e / Le
    p.s[7] = p.s[8] = 1.0 / (0.5 + nu_e / p.cs2)
    p.zeta[1] = p.zeta[2] = 1.0 / (0.5 + p.alpha_e / p.csT2)
    p.eta[1] = p.eta[2] = 1.0 / (0.5 + p.D_e / p.csT2)
    p.gbT = Gr * p.nu * p.nu / L ** 3
    p.gbC = N * p.gbT
    p.scalar_lr, p.scalar_tb = ADIABATIC, DIRICHLET
    for k, v in enumerate((0.5, 0.5, 0.0, 1.0)):
        p.Tw[k] = p.Cw[k] = v
    p.uw[3][0] = U0
    return p


def derive_convective(Nx, Ra, Da, eps, Pr, Le, N, BiT, BiC, J=1.0, sigma=1.0, Ma=0.1,
                      varpi=0.4) -> Params:
    """Porous cavity with a freely convective wall (Sec. 4.2): Nx lattice spacings
    per side (Nx + 1 nodes on walls), left wall T = C = 1, right wall convective
    (Eq. 39) to the ambient T = C = 0 with Biot numbers BiT, BiC, top and bottom
    adiabatic and impermeable; T0 = C0 = 1/2, dT = dC = 1."""
    p = derive(Nx + 1, Nx + 1, Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi, nee=True)
    p.BiT[1], p.BiC[1] = BiT, BiC
    return p


def to_model_a(p: Params) -> Params:
    """Switch p to the coupled equilibria of Eqs. 30-31 keeping the same effective
    diffusivities: by Eq. 32 alpha_e = sigma c_sT^2 (1/zeta_a - 1/2) and
    D_e = eps c_sT^2 (1/eta_D - 1/2), so the rates are re-derived from Eq. 29's."""
    za, eD = p.zeta[1], p.eta[1]
    za_a = 1.0 / (0.5 + (1.0 / za - 0.5) / p.sigma)
    eD_a = 1.0 / (0.5 + (1.0 / eD - 0.5) / p.eps)
    p.zeta[1] = p.zeta[2] = za_a
    p.eta[1] = p.eta[2] = eD_a
    p.model_a = 1
    return p


def residual_fields(now, prev):
    """Steady-state residual of Sec. 4's steady runs (reading: the relative change of
    (u_x, u_y, T, C)): now / prev are arrays [4, ...] of those fields.  Returns
    (r, diverged)."""
    a = np.ascontiguousarray(now, dtype=np.float64)
    b = np.ascontiguousarray(prev, dtype=np.float64)
    assert a.shape == b.shape and a.shape[0] == 4
    r = C.c_double()
    bad = lib().or_residual_fields(a.size // 4, _ptr(a), _ptr(b), C.byref(r))
    return r.value, bool(bad)


def noise_window(seed, noise, nx, ny, x0, y0, w, h):
    """Initial (T, C) of the window [x0, x0 + w) x [y0, y0 + h) of an nx x ny cavity with
    the seeded noise (the keys of the whole cavity), as [h][w] arrays."""
    T = np.empty((h, w))
    Cc = np.empty((h, w))
    lib().or_noise_window(C.c_uint64(seed), float(noise), int(nx), int(ny), int(x0), int(y0),
                          int(w), int(h), _ptr(T), _ptr(Cc))
    return T, Cc


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def uniform(seed: int, k: int) -> float:
    return float(lib().or_uniform(C.c_uint64(seed), C.c_uint64(k)))


class Oracle:
    """One cavity state advanced by the FP64 oracle."""

    def __init__(self, p: Params, seed: int = 1, noise: float = 1e-3, T_init=None, C_init=None,
                 eps_field=None, K_field=None):
        self.p = p
        self.nx, self.ny = p.nx, p.ny
        arr = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
               for a in (T_init, C_init, eps_field, K_field)]
        self._keep = arr
        self.h = lib().or_create_field(C.byref(p), C.c_uint64(seed), noise, *[_ptr(a) for a in arr])
        if not self.h:
            raise MemoryError("or_create failed")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    @property
    def t(self) -> int:
        return int(lib().or_time(self.h))

    def step(self, n: int = 1) -> None:
        lib().or_step(self.h, int(n))

    def fields(self):
        shp = (self.ny, self.nx)
        ux, uy, T, Cc, rho = (np.empty(shp) for _ in range(5))
        lib().or_fields(self.h, _ptr(ux), _ptr(uy), _ptr(T), _ptr(Cc), _ptr(rho))
        return {"ux": ux, "uy": uy, "T": T, "C": Cc, "rho": rho}

    def nusselt_sherwood(self) -> np.ndarray:
        out = np.empty(4)
        lib().or_nusselt_sherwood(self.h, _ptr(out))
        return out

    def nusselt_sherwood_tb(self) -> np.ndarray:
        out = np.empty(4)
        lib().or_nusselt_sherwood_tb(self.h, _ptr(out))
        return out

    def stream_function(self) -> np.ndarray:
        psi = np.empty((self.ny, self.nx))
        lib().or_stream_function(self.h, _ptr(psi))
        return psi

    def residual(self):
        """Residual of the current fields against those of the previous call (+inf on
        the first call); returns (r, diverged)."""
        if not hasattr(self, "_snap"):
            self._snap = np.zeros((4, self.ny, self.nx))
            self._have_snap = 0
        r = C.c_double()
        bad = lib().or_residual(self.h, _ptr(self._snap), self._have_snap, C.byref(r))
        self._have_snap = 1
        return r.value, bool(bad)

    def get(self):
        shp = (self.ny, self.nx)
        f = np.empty((9,) + shp)
        g = np.empty((5,) + shp)
        h = np.empty((5,) + shp)
        hist = np.empty((4,) + shp)
        lib().or_get(self.h, _ptr(f), _ptr(g), _ptr(h), _ptr(hist))
        return f, g, h, hist

    def set(self, f=None, g=None, h=None, hist=None):
        a = [None if x is None else np.ascontiguousarray(x, dtype=np.float64) for x in (f, g, h, hist)]
        lib().or_set(self.h, *[_ptr(x) for x in a])


def collide_node(p: Params, f, g, h, hist):
    """Collision of one node (Eqs. 10, 21, 22); returns f*, g*, h*, new hist, macro."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    hist = np.array(hist, dtype=np.float64)
    fs, gs, hs, mac = np.empty(9), np.empty(5), np.empty(5), np.empty(7)
    lib().or_collide_node(C.byref(p), _ptr(f), _ptr(g), _ptr(h), _ptr(hist), _ptr(fs),
                          _ptr(gs), _ptr(hs), _ptr(mac))
    return fs, gs, hs, hist, dict(zip(["rho", "ux", "uy", "T", "C", "Fx", "Fy"], mac))
