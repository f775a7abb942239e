"""ctypes binding of the C ABI in ``include/mclbm.h``.

Argument marshalling only: every step of the method runs in the CUDA
library ``_lib/libmclbm.so``.  Functions keep the C names; buffers may be
numpy arrays (host) or torch tensors (host or CUDA), and must be contiguous
with the dtype the C signature names.  There is no CPU fallback: if the
library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import build as _build

MCLBM_OK = 0
MCLBM_ERR_ARG = -1
MCLBM_ERR_CUDA = -2
MCLBM_ERR_DIVERGED = -3
MCLBM_ERR_TIMEOUT = -4
MCLBM_ERR_STATE = -5
MCLBM_ERR_NOMEM = -6

MCLBM_FP64, MCLBM_FP32, MCLBM_FP32_DEV, MCLBM_FP16_DEV, MCLBM_BF16_DEV = range(5)
PRECISIONS = {"fp64": MCLBM_FP64, "fp32": MCLBM_FP32, "fp32dev": MCLBM_FP32_DEV,
              "fp16dev": MCLBM_FP16_DEV, "bf16dev": MCLBM_BF16_DEV}
STORE_BYTES = {MCLBM_FP64: 8, MCLBM_FP32: 4, MCLBM_FP32_DEV: 4, MCLBM_FP16_DEV: 2,
               MCLBM_BF16_DEV: 2}

MCLBM_FLAG_PERIODIC_Y = 0
MCLBM_FLAG_VEL_SHIFT = 1
MCLBM_FLAG_DIAG_EVERY = 2
MCLBM_FLAG_KERNEL = 3
MCLBM_FLAG_TILE_SHAPE = 4
MCLBM_FLAG_WAIT_LIMIT_US = 5
MCLBM_FLAG_TEST_NO_COPY = 6

DIAG_FIELDS = ("mass1", "mass2", "sw_count", "sw_mass", "p_in", "p_out", "pc", "n_fluid")


class CaseDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("solid", C.c_void_p), ("xi", C.c_void_p),
                ("nu1", C.c_double), ("nu2", C.c_double), ("g_coh", C.c_double),
                ("g_ads", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
                ("rho_in1", C.c_double), ("rho_out2", C.c_double), ("periodic_y", C.c_int),
                ("rho1", C.c_void_p), ("rho2", C.c_void_p)]


class MclbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mclbm error {code}: {msg}")
        self.code = code


_lib = None
_P = C.POINTER
_vp = C.c_void_p
_i64 = C.c_int64

_SIGS = {
    "mclbm_create": (C.c_int, [C.c_int, C.c_int, _vp, _vp, C.c_int, _vp, _P(_vp)]),
    "mclbm_destroy": (C.c_int, [_vp]),
    "mclbm_set_flag": (C.c_int, [_vp, C.c_int, _i64]),
    "mclbm_set_viscosity": (C.c_int, [_vp, C.c_double, C.c_double]),
    "mclbm_set_coupling": (C.c_int, [_vp, C.c_double, C.c_double]),
    "mclbm_set_body_force": (C.c_int, [_vp, C.c_double, C.c_double]),
    "mclbm_set_pressure_bc": (C.c_int, [_vp, C.c_double, C.c_double]),
    "mclbm_set_pressure_bc_p": (C.c_int, [_vp, C.c_double, C.c_double]),
    "mclbm_set_bc": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double]),
    "mclbm_set_mrt": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, C.c_double]),
    "mclbm_set_stream": (C.c_int, [_vp, _vp]),
    "mclbm_init_densities": (C.c_int, [_vp, _vp, _vp]),
    "mclbm_set_populations": (C.c_int, [_vp, _vp]),
    "mclbm_get_populations": (C.c_int, [_vp, _vp]),
    "mclbm_step": (C.c_int, [_vp, _i64]),
    "mclbm_synchronize": (C.c_int, [_vp]),
    "mclbm_read_density": (C.c_int, [_vp, C.c_int, _vp]),
    "mclbm_read_velocity": (C.c_int, [_vp, _vp, _vp]),
    "mclbm_read_pressure": (C.c_int, [_vp, _vp]),
    "mclbm_read_phase": (C.c_int, [_vp, _vp]),
    "mclbm_diagnostics": (C.c_int, [_vp, _vp]),
    "mclbm_saturation": (C.c_int, [_vp, _P(C.c_double), _P(C.c_double)]),
    "mclbm_capillary_pressure": (C.c_int, [_vp, _P(C.c_double), _P(C.c_double), _P(C.c_double)]),
    "mclbm_mass": (C.c_int, [_vp, _vp]),
    "mclbm_info": (C.c_int, [_vp, _vp]),
    "mclbm_batch_create": (C.c_int, [C.c_int, _vp, C.c_int, _vp, _P(_vp)]),
    "mclbm_batch_destroy": (C.c_int, [_vp]),
    "mclbm_batch_lattice": (C.c_int, [_vp, C.c_int, _P(_vp)]),
    "mclbm_batch_step": (C.c_int, [_vp, _i64]),
    "mclbm_batch_info": (C.c_int, [_vp, _vp]),
    "mclbm_batch_tuning": (C.c_int, [_vp, _vp]),
    "mclbm_diagnostics_noalloc": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_double, C.c_int,
                                            _vp, _vp]),
    "mclbm_unet_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _P(_vp)]),
    "mclbm_unet_destroy": (C.c_int, [_vp]),
    "mclbm_unet_param_count": (C.c_int, [_vp, _P(_i64)]),
    "mclbm_unet_set_max_ctas": (C.c_int, [_vp, C.c_int]),
    "mclbm_unet_set_shared_taps": (C.c_int, [_vp, C.c_int]),
    "mclbm_unet_set_params": (C.c_int, [_vp, _vp]),
    "mclbm_unet_get_params": (C.c_int, [_vp, _vp]),
    "mclbm_unet_infer": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "mclbm_unet_gradient": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp,
                                      _P(C.c_double), _vp]),
    "mclbm_unet_train_step": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp,
                                        C.c_double, _P(C.c_double)]),
    "mclbm_init_from_phase": (C.c_int, [_vp, _vp]),
    "mclbm_blend_phase": (C.c_int, [_vp, _vp, C.c_double, _P(_i64)]),
    "mclbm_fluid_layout_check": (C.c_int, [C.c_int, C.c_int, _vp, C.c_int, C.c_int, C.c_int, _vp]),
    "mclbm_save": (C.c_int, [_vp, C.c_char_p]),
    "mclbm_load": (C.c_int, [_vp, C.c_char_p]),
    "mclbm_launch_count": (_i64, []),
    "mclbm_last_error": (C.c_char_p, []),
}


def library_path() -> Path:
    return _build.LIB


def load(build: bool = True):
    """Load libmclbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    path = library_path()
    if not path.exists():
        raise RuntimeError(f"CUDA library {path} is missing; run the package build first")
    lib = C.CDLL(str(path))
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != MCLBM_OK:
        msg = load().mclbm_last_error()
        raise MclbmError(rc, msg.decode() if msg else "")


def _addr(buf, dtype) -> int:
    """Address of a contiguous numpy array or torch tensor of the given dtype."""
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {buf.dtype}")
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data
    # torch tensor
    import torch
    want = {np.float64: torch.float64, np.float32: torch.float32,
            np.uint8: torch.uint8}[np.dtype(dtype).type]
    if buf.dtype != want:
        raise TypeError(f"expected {want}, got {buf.dtype}")
    if not buf.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return buf.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# --- the C functions, same names -------------------------------------------------

def mclbm_create(nx: int, ny: int, solid, xi=None, prec: int = MCLBM_FP32, stream=None):
    lib = load()
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    if solid.shape != (ny, nx):
        raise ValueError(f"solid must be [ny][nx] = [{ny}][{nx}]")
    xi_arr = None if xi is None else np.ascontiguousarray(xi, dtype=np.float32)
    if xi_arr is not None and xi_arr.shape != (ny, nx):
        raise ValueError("xi must be [ny][nx]")
    h = _vp()
    _check(lib.mclbm_create(nx, ny, _addr(solid, np.uint8), _addr(xi_arr, np.float32),
                            int(prec), _stream_handle(stream), C.byref(h)))
    return h


def mclbm_destroy(h) -> None:
    _check(load().mclbm_destroy(h))


def mclbm_set_flag(h, flag: int, value: int) -> None:
    _check(load().mclbm_set_flag(h, flag, int(value)))


def mclbm_set_viscosity(h, nu1: float, nu2: float) -> None:
    _check(load().mclbm_set_viscosity(h, nu1, nu2))


def mclbm_set_coupling(h, g_coh: float, g_ads: float) -> None:
    _check(load().mclbm_set_coupling(h, g_coh, g_ads))


def mclbm_set_body_force(h, gx: float, gy: float) -> None:
    _check(load().mclbm_set_body_force(h, gx, gy))


def mclbm_set_pressure_bc(h, rho_in1: float, rho_out2: float) -> None:
    _check(load().mclbm_set_pressure_bc(h, rho_in1, rho_out2))


def mclbm_set_mrt(h, on: bool, s_e: float = 0.0, s_eps: float = 0.0, s_q: float = 0.0) -> None:
    _check(load().mclbm_set_mrt(h, int(bool(on)), float(s_e), float(s_eps), float(s_q)))


def mclbm_set_bc(h, bc_set: int, rho_in2: float = 0.0, rho_out1: float = 0.0) -> None:
    _check(load().mclbm_set_bc(h, int(bc_set), float(rho_in2), float(rho_out1)))


def mclbm_set_pressure_bc_p(h, p_in: float, p_out: float) -> None:
    _check(load().mclbm_set_pressure_bc_p(h, p_in, p_out))


def mclbm_set_stream(h, stream) -> None:
    _check(load().mclbm_set_stream(h, _stream_handle(stream)))


def mclbm_init_densities(h, rho1, rho2) -> None:
    _check(load().mclbm_init_densities(h, _addr(rho1, np.float64), _addr(rho2, np.float64)))


def mclbm_save(h, path) -> None:
    _check(load().mclbm_save(h, str(path).encode()))


def mclbm_load(h, path) -> None:
    _check(load().mclbm_load(h, str(path).encode()))


def mclbm_init_from_phase(h, phi) -> None:
    _check(load().mclbm_init_from_phase(h, _addr(phi, np.float32)))


def mclbm_blend_phase(h, phi_hat, flip: float = 0.0) -> int:
    """Warm start in place from a predicted phase field [ny][nx] (float32,
    host or device); returns the number of nodes reset."""
    n = C.c_int64(0)
    _check(load().mclbm_blend_phase(h, _addr(phi_hat, np.float32), float(flip), C.byref(n)))
    return int(n.value)


def mclbm_set_populations(h, f) -> None:
    _check(load().mclbm_set_populations(h, _addr(f, np.float64)))


def mclbm_get_populations(h, f) -> None:
    _check(load().mclbm_get_populations(h, _addr(f, np.float64)))


def mclbm_step(h, nsteps: int) -> None:
    _check(load().mclbm_step(h, int(nsteps)))


def mclbm_synchronize(h) -> None:
    _check(load().mclbm_synchronize(h))


def mclbm_read_density(h, comp: int, out) -> None:
    _check(load().mclbm_read_density(h, comp, _addr(out, np.float64)))


def mclbm_read_velocity(h, ux, uy) -> None:
    _check(load().mclbm_read_velocity(h, _addr(ux, np.float64), _addr(uy, np.float64)))


def mclbm_read_pressure(h, out) -> None:
    _check(load().mclbm_read_pressure(h, _addr(out, np.float64)))


def mclbm_read_phase(h, out) -> None:
    _check(load().mclbm_read_phase(h, _addr(out, np.float32)))


def mclbm_diagnostics(h) -> dict:
    out = np.zeros(8)
    _check(load().mclbm_diagnostics(h, out.ctypes.data))
    return dict(zip(DIAG_FIELDS, out.tolist()))


def mclbm_saturation(h) -> tuple[float, float]:
    a, b = C.c_double(), C.c_double()
    _check(load().mclbm_saturation(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def mclbm_capillary_pressure(h) -> tuple[float, float, float]:
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(load().mclbm_capillary_pressure(h, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def mclbm_mass(h) -> tuple[float, float]:
    out = np.zeros(2)
    _check(load().mclbm_mass(h, out.ctypes.data))
    return float(out[0]), float(out[1])


def mclbm_info(h) -> dict:
    out = np.zeros(6, dtype=np.int64)
    _check(load().mclbm_info(h, out.ctypes.data))
    return dict(zip(("nx", "ny", "pitch", "precision", "steps", "device_bytes"), out.tolist()))


def mclbm_diagnostics_noalloc(f, solid, nx: int, ny: int, g_coh: float, periodic_y: bool,
                              out, stream=None) -> None:
    """Diagnostics of caller-owned device populations [2][9][ny][nx] and
    solid mask [ny][nx], without any allocation (see include/mclbm.h); out
    is a [8] float64 buffer on the device or the host.  The buffer sizes are
    checked here: the library reads 18 * nx * ny doubles of f and nx * ny
    bytes of solid through raw pointers and cannot check them itself."""
    n = int(nx) * int(ny)
    for buf, need, name in ((f, 18 * n, "f"), (solid, n, "solid"), (out, 8, "out")):
        have = buf.size if isinstance(buf, np.ndarray) else buf.numel()
        if have < need:
            raise ValueError(f"{name} holds {have} elements, needs at least {need}")
    _check(load().mclbm_diagnostics_noalloc(_addr(f, np.float64), _addr(solid, np.uint8),
                                            int(nx), int(ny), float(g_coh), int(periodic_y),
                                            _addr(out, np.float64), _stream_handle(stream)))


def mclbm_batch_create(cases: list[dict], prec: int = MCLBM_FP32, stream=None):
    """cases: dicts with solid, xi, nu1, nu2, g_coh, g_ads, gx, gy, rho_in1,
    rho_out2, periodic_y, rho1, rho2 (numpy host arrays)."""
    lib = load()
    keep = []
    arr = (CaseDesc * len(cases))()
    for d, c in zip(arr, cases):
        solid = np.ascontiguousarray(c["solid"], dtype=np.uint8)
        ny, nx = solid.shape
        xi = np.ascontiguousarray(c.get("xi", np.zeros((ny, nx))), dtype=np.float32)
        r1 = np.ascontiguousarray(c["rho1"], dtype=np.float64)
        r2 = np.ascontiguousarray(c["rho2"], dtype=np.float64)
        keep += [solid, xi, r1, r2]
        d.nx, d.ny = nx, ny
        d.solid, d.xi = solid.ctypes.data, xi.ctypes.data
        d.nu1, d.nu2 = c.get("nu1", 1 / 6), c.get("nu2", 1 / 6)
        d.g_coh = c.get("g_coh", 3.5)
        d.g_ads = c.get("g_ads", d.g_coh)
        d.gx, d.gy = c.get("gx", 0.0), c.get("gy", 0.0)
        d.rho_in1, d.rho_out2 = c.get("rho_in1", -1.0), c.get("rho_out2", -1.0)
        d.periodic_y = int(c.get("periodic_y", False))
        d.rho1, d.rho2 = r1.ctypes.data, r2.ctypes.data
    h = _vp()
    _check(lib.mclbm_batch_create(len(cases), C.cast(arr, _vp), int(prec),
                                  _stream_handle(stream), C.byref(h)))
    return h


def mclbm_batch_destroy(b) -> None:
    _check(load().mclbm_batch_destroy(b))


def mclbm_batch_lattice(b, k: int):
    h = _vp()
    _check(load().mclbm_batch_lattice(b, int(k), C.byref(h)))
    return h


def mclbm_batch_step(b, nsteps: int) -> None:
    _check(load().mclbm_batch_step(b, int(nsteps)))


def mclbm_batch_info(b) -> dict:
    out = np.zeros(8, dtype=np.int64)
    _check(load().mclbm_batch_info(b, out.ctypes.data))
    return dict(zip(("cases", "nodes", "shape", "grid", "graph_steps", "steps", "slots",
                     "graph"), out.tolist()))


def mclbm_batch_tuning(b) -> list[float]:
    out = np.zeros(6)
    _check(load().mclbm_batch_tuning(b, out.ctypes.data))
    return out.tolist()


def mclbm_fluid_layout_check(codes, prec: str = "fp32", tile_shape: int = 0, open_x: bool = False) -> dict:
    """Build and check the fluid-only layout on the host (no GPU) for
    geometry codes of shape (ny + 6, nx + 6) (see include/mclbm.h)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    if codes.ndim != 2 or codes.shape[0] < 7 or codes.shape[1] < 7:
        raise ValueError("codes must be a (ny + 6, nx + 6) array")
    ny, nx = codes.shape[0] - 6, codes.shape[1] - 6
    out = np.zeros(8, dtype=np.int64)
    _check(load().mclbm_fluid_layout_check(nx, ny, codes.ctypes.data, PRECISIONS[prec], int(tile_shape),
                                           int(open_x), out.ctypes.data))
    keys = ("tiles", "slots", "max_stage", "table_words", "attempts", "max_own", "smem_bytes", "check")
    return dict(zip(keys, out.tolist()))


def mclbm_launch_count() -> int:
    return int(load().mclbm_launch_count())


def mclbm_last_error() -> str:
    msg = load().mclbm_last_error()
    return msg.decode() if msg else ""


# --- a small object wrapper ---------------------------------------------------------

class Lattice:
    """Owning handle of one lattice (context manager)."""

    def __init__(self, solid, xi=None, *, prec: int | str = MCLBM_FP32, nu1: float = 1 / 6,
                 nu2: float = 1 / 6, g_coh: float = 3.5, g_ads: float | None = None,
                 rho_in1: float = -1.0, rho_out2: float = -1.0, periodic_y: bool = False,
                 vel_shift: bool = True, gx: float = 0.0, gy: float = 0.0, stream=None,
                 kernel: int = 0, tile_shape: int = 0, bc_set: int = 3, rho_in2: float = 0.0,
                 rho_out1: float = 0.0, mrt: bool = False, s_e: float = 0.0, s_eps: float = 0.0,
                 s_q: float = 0.0):
        self.h = None
        if isinstance(prec, str):
            prec = PRECISIONS[prec]
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.ny, self.nx = solid.shape
        self.prec = prec
        self.h = mclbm_create(self.nx, self.ny, solid, xi, prec, stream)
        mclbm_set_viscosity(self.h, nu1, nu2)
        mclbm_set_coupling(self.h, g_coh, g_coh if g_ads is None else g_ads)
        mclbm_set_pressure_bc(self.h, rho_in1, rho_out2)
        mclbm_set_bc(self.h, bc_set, rho_in2, rho_out1)
        mclbm_set_mrt(self.h, mrt, s_e, s_eps, s_q)
        mclbm_set_flag(self.h, MCLBM_FLAG_PERIODIC_Y, int(periodic_y))
        mclbm_set_flag(self.h, MCLBM_FLAG_VEL_SHIFT, int(vel_shift))
        mclbm_set_body_force(self.h, gx, gy)
        mclbm_set_flag(self.h, MCLBM_FLAG_KERNEL, kernel)
        mclbm_set_flag(self.h, MCLBM_FLAG_TILE_SHAPE, tile_shape)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            mclbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, rho1, rho2) -> None:
        r1 = rho1 if not isinstance(rho1, np.ndarray) else np.ascontiguousarray(rho1, np.float64)
        r2 = rho2 if not isinstance(rho2, np.ndarray) else np.ascontiguousarray(rho2, np.float64)
        mclbm_init_densities(self.h, r1, r2)

    def step(self, n: int = 1) -> None:
        mclbm_step(self.h, n)

    def sync(self) -> None:
        mclbm_synchronize(self.h)

    def populations(self) -> np.ndarray:
        f = np.zeros((2, 9, self.ny, self.nx))
        mclbm_get_populations(self.h, f)
        return f

    def set_populations(self, f) -> None:
        mclbm_set_populations(self.h, np.ascontiguousarray(f, dtype=np.float64))

    def density(self) -> np.ndarray:
        out = np.zeros((2, self.ny, self.nx))
        mclbm_read_density(self.h, 1, out[0])
        mclbm_read_density(self.h, 2, out[1])
        return out

    def velocity(self):
        ux = np.zeros((self.ny, self.nx))
        uy = np.zeros((self.ny, self.nx))
        mclbm_read_velocity(self.h, ux, uy)
        return ux, uy

    def pressure(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx))
        mclbm_read_pressure(self.h, out)
        return out

    def phase(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx), dtype=np.float32)
        mclbm_read_phase(self.h, out)
        return out

    def diagnostics(self) -> dict:
        return mclbm_diagnostics(self.h)

    def set_pressure_bc(self, rho_in1: float, rho_out2: float) -> None:
        mclbm_set_pressure_bc(self.h, rho_in1, rho_out2)

    def set_bc(self, bc_set: int, rho_in2: float = 0.0, rho_out1: float = 0.0) -> None:
        mclbm_set_bc(self.h, bc_set, rho_in2, rho_out1)

    def set_mrt(self, on: bool, s_e: float = 0.0, s_eps: float = 0.0, s_q: float = 0.0) -> None:
        mclbm_set_mrt(self.h, on, s_e, s_eps, s_q)

    def info(self) -> dict:
        return mclbm_info(self.h)


class LatticeView(Lattice):
    """A borrowed case of a batch: parameters and read-outs, not stepping."""

    def __init__(self, batch, k: int, ny: int, nx: int, prec: int):
        self.h = mclbm_batch_lattice(batch, k)
        self.ny, self.nx, self.prec = ny, nx, prec

    def close(self) -> None:  # owned by the batch
        self.h = None

    def step(self, n: int = 1) -> None:
        raise RuntimeError("a batch case is stepped with mclbm_batch_step")


# --- learned warm start ----------------------------------------------------------

def mclbm_unet_create(levels: int, base: int, max_batch: int, max_h: int, max_w: int, stream=None):
    h = _vp()
    _check(load().mclbm_unet_create(levels, base, max_batch, max_h, max_w, _stream_handle(stream),
                                    C.byref(h)))
    return h


def mclbm_unet_destroy(h) -> None:
    _check(load().mclbm_unet_destroy(h))


def mclbm_unet_param_count(h) -> int:
    n = _i64()
    _check(load().mclbm_unet_param_count(h, C.byref(n)))
    return n.value


def mclbm_unet_set_max_ctas(h, n: int) -> None:
    _check(load().mclbm_unet_set_max_ctas(h, int(n)))


def mclbm_unet_set_shared_taps(h, enable: int) -> None:
    _check(load().mclbm_unet_set_shared_taps(h, int(enable)))


def mclbm_unet_set_params(h, theta) -> None:
    _check(load().mclbm_unet_set_params(h, _addr(theta, np.float32)))


def mclbm_unet_get_params(h, theta) -> None:
    _check(load().mclbm_unet_get_params(h, _addr(theta, np.float32)))


def mclbm_unet_infer(h, batch: int, height: int, width: int, x, phi) -> None:
    _check(load().mclbm_unet_infer(h, batch, height, width, _addr(x, np.float32),
                                   _addr(phi, np.float32)))


def mclbm_unet_gradient(h, batch: int, height: int, width: int, x, target, mask, grad=None) -> float:
    loss = C.c_double()
    _check(load().mclbm_unet_gradient(h, batch, height, width, _addr(x, np.float32),
                                      _addr(target, np.float32), _addr(mask, np.float32),
                                      C.byref(loss), _addr(grad, np.float32)))
    return loss.value


def mclbm_unet_train_step(h, batch: int, height: int, width: int, x, target, mask,
                          lr: float) -> float:
    loss = C.c_double()
    _check(load().mclbm_unet_train_step(h, batch, height, width, _addr(x, np.float32),
                                        _addr(target, np.float32), _addr(mask, np.float32),
                                        float(lr), C.byref(loss)))
    return loss.value


class UNet:
    """Owning handle of a warm-start network (arrays NHWC, FP32)."""

    def __init__(self, levels: int = 4, base: int = 32, max_batch: int = 1, max_h: int = 256,
                 max_w: int = 256, stream=None):
        self.h = None
        self.levels, self.base = levels, base
        self.h = mclbm_unet_create(levels, base, max_batch, max_h, max_w, stream)
        self.n = mclbm_unet_param_count(self.h)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            mclbm_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_params(self, theta) -> None:
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        if theta.size != self.n:
            raise ValueError(f"expected {self.n} parameters, got {theta.size}")
        mclbm_unet_set_params(self.h, theta)

    def params(self) -> np.ndarray:
        out = np.empty(self.n, np.float32)
        mclbm_unet_get_params(self.h, out)
        return out

    def infer(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        b, hh, ww, _ = x.shape
        out = np.empty((b, hh, ww), np.float32)
        mclbm_unet_infer(self.h, b, hh, ww, x, out)
        return out

    def gradient(self, x, target, mask):
        x = np.ascontiguousarray(x, dtype=np.float32)
        b, hh, ww, _ = x.shape
        g = np.empty(self.n, np.float32)
        loss = mclbm_unet_gradient(self.h, b, hh, ww, x, np.ascontiguousarray(target, np.float32),
                                   np.ascontiguousarray(mask, np.float32), g)
        return loss, g

    def train_step(self, x, target, mask, lr: float) -> float:
        x = np.ascontiguousarray(x, dtype=np.float32)
        b, hh, ww, _ = x.shape
        return mclbm_unet_train_step(self.h, b, hh, ww, x, np.ascontiguousarray(target, np.float32),
                                     np.ascontiguousarray(mask, np.float32), lr)
