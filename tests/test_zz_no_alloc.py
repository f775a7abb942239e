"""The allocation-free diagnostics entry point, for callers that cannot call
cudaMalloc (their device memory comes from their own pool, or they must not
allocate once running).  It must give the same results as the lattice's
own diagnostics on the same populations, call after call, although every
call reuses one fixed scratch array inside the library.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import math

import numpy as np
import pytest

from paper_2111_08666_gb300 import mclbm, media

pytestmark = pytest.mark.gpu


def _compare(got, ref):
    for k, name in enumerate(mclbm.DIAG_FIELDS):
        a, b = float(got[k]), ref[name]
        if math.isnan(b):
            assert math.isnan(a), name
        elif name in ("sw_count", "n_fluid"):
            assert a == b, name
        elif name == "pc":           # a difference of two ~0.37 pressures
            assert a == pytest.approx(b, abs=1e-13), name
        else:
            assert a == pytest.approx(b, rel=1e-12, abs=1e-14), name


def test_noalloc_diagnostics_match_lattice_diagnostics_twice():
    import torch
    torch.cuda.set_device(0)
    c = media.config_small_fp64()
    lat = mclbm.Lattice(c["solid"], media.uniform_xi(c["solid"], -0.4), prec="fp64",
                        nu1=c["nu1"], nu2=c["nu2"], rho_in1=c["rho_in1"], rho_out2=c["rho_out2"])
    lat.init(c["rho1"], c["rho2"])
    ny, nx = c["solid"].shape
    solid_dev = torch.from_numpy(np.ascontiguousarray(c["solid"])).cuda()
    f_dev = torch.empty((2, 9, ny, nx), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call, steps in enumerate((120, 80)):
        lat.step(steps)
        mclbm.mclbm_get_populations(lat.h, f_dev)
        ref = lat.diagnostics()
        # device output, then host output
        out_dev = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        mclbm.mclbm_diagnostics_noalloc(f_dev, solid_dev, nx, ny, 3.5, False, out_dev, stream)
        torch.cuda.synchronize()
        _compare(out_dev.cpu().numpy(), ref)
        out_host = np.full(8, np.nan)
        mclbm.mclbm_diagnostics_noalloc(f_dev, solid_dev, nx, ny, 3.5, False, out_host, stream)
        _compare(out_host, ref)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    """The size limit is checked by the library itself (called here through
    the C ABI directly: the binding would first refuse buffers this small
    for a 4096 x 2048 lattice), before any kernel reads the buffers."""
    import torch
    f_dev = torch.zeros(18, dtype=torch.float64, device="cuda")
    solid_dev = torch.zeros(1, dtype=torch.uint8, device="cuda")
    out = np.zeros(8)
    lib = mclbm.load()
    rc = lib.mclbm_diagnostics_noalloc(f_dev.data_ptr(), solid_dev.data_ptr(), 4096, 2048, 3.5, 0,
                                       out.ctypes.data, None)
    assert rc == mclbm.MCLBM_ERR_ARG
    assert b"static scratch" in lib.mclbm_last_error()
    with pytest.raises(ValueError):
        mclbm.mclbm_diagnostics_noalloc(f_dev, solid_dev, 4096, 2048, 3.5, False, out)
