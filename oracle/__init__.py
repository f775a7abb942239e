"""ctypes wrapper and build step of the FP64 CPU oracle (``mclbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use this module to produce reference results.  The CUDA
library and its Python binding never import it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "mclbm_oracle.c"
_LIB_DIR = _HERE / "_lib"
_LIB = _LIB_DIR / "liboracle.so"

# number of values returned by oracle_diagnostics
DIAG_FIELDS = ("mass1", "mass2", "sw_count", "sw_mass", "p_in", "p_out", "pc", "n_fluid")


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("nu1", C.c_double), ("nu2", C.c_double),
                ("g_coh", C.c_double), ("g_ads", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double),
                ("rho_in1", C.c_double), ("rho_out2", C.c_double),
                ("open_x", C.c_int), ("periodic_y", C.c_int),
                ("vel_shift", C.c_int), ("bc_set", C.c_int),
                ("rho_in2", C.c_double), ("rho_out1", C.c_double),
                ("mrt", C.c_int), ("pad2", C.c_int),
                ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double)]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C, OpenMP, no FMA contraction)."""
    _LIB_DIR.mkdir(exist_ok=True)
    if not force and _LIB.exists() and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    tmp = _LIB_DIR / f"liboracle.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_LIB))
        P = C.POINTER
        dp, fp, u8p = P(C.c_double), P(C.c_float), P(C.c_uint8)
        L.oracle_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.oracle_source.argtypes = [C.c_double] * 4 + [dp]
        L.oracle_pressure.argtypes = [C.c_double] * 3
        L.oracle_pressure.restype = C.c_double
        L.oracle_init.argtypes = [P(Params), u8p, dp, dp, dp, dp]
        L.oracle_stream_bc.argtypes = [P(Params), u8p, dp, dp, dp]
        L.oracle_moments.argtypes = [P(Params), u8p, dp, dp, dp, dp]
        L.oracle_ivsd.argtypes = [P(Params), u8p, fp, dp, dp]
        L.oracle_forces.argtypes = [P(Params), u8p, dp, dp, dp, dp]
        L.oracle_collide.argtypes = [P(Params), u8p, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.oracle_step.argtypes = [P(Params), u8p, fp, dp, dp, C.c_long, dp, dp]
        L.oracle_step.restype = C.c_int
        L.oracle_diagnostics.argtypes = [P(Params), u8p, dp, dp]
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_feq(rho, ux, uy, _ptr(out, C.c_double))
    return out


def source(ux: float, uy: float, fx: float, fy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_source(ux, uy, fx, fy, _ptr(out, C.c_double))
    return out


def pressure(g: float, rho1, rho2):
    return float(lib().oracle_pressure(g, float(rho1), float(rho2)))


class Oracle:
    """One lattice held in FP64 host arrays, stepped by the C oracle."""

    def __init__(self, solid: np.ndarray, xi: np.ndarray, *, nu1: float, nu2: float,
                 g_coh: float = 3.5, g_ads: float | None = None, gx: float = 0.0,
                 gy: float = 0.0, rho_in1: float = -1.0, rho_out2: float = -1.0,
                 periodic_y: bool = False, vel_shift: bool = True, bc_set: int = 3,
                 rho_in2: float = 0.0, rho_out1: float = 0.0, mrt: bool = False,
                 s_e: float = 0.0, s_eps: float = 0.0, s_q: float = 0.0):
        self.solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.ny, self.nx = self.solid.shape
        self.xi = np.ascontiguousarray(xi, dtype=np.float32)
        open_x = rho_in1 >= 0 and rho_out2 >= 0
        self.p = Params(self.nx, self.ny, nu1, nu2, g_coh,
                        g_coh if g_ads is None else g_ads, gx, gy,
                        rho_in1, rho_out2, int(open_x), int(periodic_y),
                        int(vel_shift), int(bc_set), rho_in2, rho_out1, int(mrt), 0,
                        s_e, s_eps, s_q)
        self.f = np.zeros((2, 9, self.ny, self.nx))
        # frozen boundary values: component 1's outlet f_{3,6,7} (Eq. 26, rows
        # 0-2) and component 2's inlet f_{1,5,8} (Eq. 27, rows 3-5)
        self.d5 = np.zeros((6, self.ny))
        self.ux = np.zeros((self.ny, self.nx))
        self.uy = np.zeros((self.ny, self.nx))
        self.steps = 0

    def set_bc(self, bc_set: int, rho_in2: float = 0.0, rho_out1: float = 0.0) -> None:
        """Inlet/outlet treatment of Sec. 2.3: Set-1, -2 or -3; Set-1 also
        fixes component 2 at the inlet (rho_in2) and component 1 at the
        outlet (rho_out1)."""
        self.p.bc_set, self.p.rho_in2, self.p.rho_out1 = int(bc_set), rho_in2, rho_out1

    def set_mrt(self, on: bool, s_e: float = 0.0, s_eps: float = 0.0, s_q: float = 0.0) -> None:
        """MRT collision (not in the paper): rates of the energy, energy-square
        and heat-flux moments; 0 ties a rate to 1/tau_s, s_q = -1 takes
        8 (2 - w) / (8 - w)."""
        self.p.mrt, self.p.s_e, self.p.s_eps, self.p.s_q = int(on), s_e, s_eps, s_q

    def set_pressure_bc(self, rho_in1: float, rho_out2: float) -> None:
        self.p.rho_in1, self.p.rho_out2 = rho_in1, rho_out2
        self.p.open_x = int(rho_in1 >= 0 and rho_out2 >= 0)

    def init(self, rho1: np.ndarray, rho2: np.ndarray) -> None:
        r1 = np.ascontiguousarray(rho1, dtype=np.float64)
        r2 = np.ascontiguousarray(rho2, dtype=np.float64)
        lib().oracle_init(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                          _ptr(r1, C.c_double), _ptr(r2, C.c_double),
                          _ptr(self.f, C.c_double), _ptr(self.d5, C.c_double))
        self.steps = 0

    def step(self, n: int = 1) -> None:
        rc = lib().oracle_step(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                               _ptr(self.xi, C.c_float), _ptr(self.d5, C.c_double),
                               _ptr(self.f, C.c_double), int(n),
                               _ptr(self.ux, C.c_double), _ptr(self.uy, C.c_double))
        if rc != 0:
            raise MemoryError("oracle_step could not allocate")
        self.steps += n

    # individual steps of one update, for the pins
    def stream_bc(self, fpost: np.ndarray | None = None) -> np.ndarray:
        src = self.f if fpost is None else np.ascontiguousarray(fpost)
        out = np.zeros_like(self.f)
        lib().oracle_stream_bc(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                               _ptr(self.d5, C.c_double), _ptr(src, C.c_double),
                               _ptr(out, C.c_double))
        return out

    def moments(self, f: np.ndarray):
        f = np.ascontiguousarray(f)
        rho = np.zeros((2, self.ny, self.nx))
        jx = np.zeros_like(rho)
        jy = np.zeros_like(rho)
        lib().oracle_moments(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                             _ptr(f, C.c_double), _ptr(rho, C.c_double),
                             _ptr(jx, C.c_double), _ptr(jy, C.c_double))
        return rho, jx, jy

    def ivsd(self, rho: np.ndarray) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        psi = np.zeros_like(rho)
        lib().oracle_ivsd(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                          _ptr(self.xi, C.c_float), _ptr(rho, C.c_double),
                          _ptr(psi, C.c_double))
        return psi

    def forces(self, rho: np.ndarray, psi: np.ndarray):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        fx = np.zeros_like(rho)
        fy = np.zeros_like(rho)
        lib().oracle_forces(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                            _ptr(rho, C.c_double), _ptr(psi, C.c_double),
                            _ptr(fx, C.c_double), _ptr(fy, C.c_double))
        return fx, fy

    def collide(self, f, rho, jx, jy, fx, fy):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (f, rho, jx, jy, fx, fy)]
        out = np.zeros_like(self.f)
        ux = np.zeros((self.ny, self.nx))
        uy = np.zeros_like(ux)
        lib().oracle_collide(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                             *[_ptr(a, C.c_double) for a in arrs],
                             _ptr(out, C.c_double), _ptr(ux, C.c_double),
                             _ptr(uy, C.c_double))
        return out, ux, uy

    def diagnostics(self) -> dict:
        out = np.zeros(len(DIAG_FIELDS))
        lib().oracle_diagnostics(C.byref(self.p), _ptr(self.solid, C.c_uint8),
                                 _ptr(self.f, C.c_double), _ptr(out, C.c_double))
        return dict(zip(DIAG_FIELDS, out.tolist()))

    def density(self) -> np.ndarray:
        return self.f.sum(axis=1) * (self.solid == 0)

    def pressure_field(self) -> np.ndarray:
        r = self.density()
        g = self.p.g_coh
        return (r[0] + r[1]) / 3.0 + g / 3.0 * r[0] * r[1]
