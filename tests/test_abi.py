"""The C ABI library builds, loads without a GPU, exports every function the
header declares, and rejects bad arguments before touching the device."""
import ctypes as C
import re
from pathlib import Path

import pytest

from paper_2111_08666_gb300 import mclbm

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(mclbm_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mclbm_create", "mclbm_step", "mclbm_read_density", "mclbm_read_velocity",
                     "mclbm_saturation", "mclbm_capillary_pressure", "mclbm_mass",
                     "mclbm_set_pressure_bc", "mclbm_set_viscosity", "mclbm_set_coupling",
                     "mclbm_destroy", "mclbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = mclbm.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared_functions() if not hasattr(mclbm, n)]
    assert not missing, missing


def test_argument_errors_without_a_device():
    lib = mclbm.load()
    h = C.c_void_p()
    assert lib.mclbm_create(8, 8, None, None, 1, None, C.byref(h)) == mclbm.MCLBM_ERR_ARG
    assert b"solid" in lib.mclbm_last_error()
    assert lib.mclbm_create(2, 8, None, None, 1, None, C.byref(h)) == mclbm.MCLBM_ERR_ARG
    assert lib.mclbm_create(8, 8, None, None, 1, None, None) == mclbm.MCLBM_ERR_ARG
    assert lib.mclbm_step(None, 1) == mclbm.MCLBM_ERR_ARG
    assert lib.mclbm_set_viscosity(None, 0.1, 0.1) == mclbm.MCLBM_ERR_ARG
    assert lib.mclbm_destroy(None) == mclbm.MCLBM_OK
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_step(None, 1)
    assert e.value.code == mclbm.MCLBM_ERR_ARG


def test_unet_rejects_bad_shapes_without_a_device():
    lib = mclbm.load()
    h = C.c_void_p()
    for levels, base, b, hh, ww in [(0, 32, 1, 64, 64), (4, 16, 1, 64, 64), (4, 32, 0, 64, 64),
                                    (4, 32, 1, 60, 64), (7, 32, 1, 256, 256), (4, 32, 1024, 2048, 1024)]:
        rc = lib.mclbm_unet_create(levels, base, b, hh, ww, None, C.byref(h))
        assert rc == mclbm.MCLBM_ERR_ARG
        assert h.value is None


def test_unet_switches_reject_bad_arguments_without_a_device():
    lib = mclbm.load()
    assert lib.mclbm_unet_set_max_ctas(None, 4) == mclbm.MCLBM_ERR_ARG
    assert lib.mclbm_unet_set_shared_taps(None, 1) == mclbm.MCLBM_ERR_ARG
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_unet_set_shared_taps(None, 0)
    assert e.value.code == mclbm.MCLBM_ERR_ARG


def test_noalloc_binding_rejects_short_buffers_before_the_library():
    import numpy as np
    nx, ny = 16, 8
    f = np.zeros(18 * nx * ny, dtype=np.float64)
    solid = np.zeros(nx * ny, dtype=np.uint8)
    out = np.zeros(8, dtype=np.float64)
    for args, name in (((f[:-1], solid, out), "f"), ((f, solid[:-1], out), "solid"),
                       ((f, solid, out[:7]), "out")):
        with pytest.raises(ValueError, match=name):
            mclbm.mclbm_diagnostics_noalloc(args[0], args[1], nx, ny, 3.5, False, args[2])
