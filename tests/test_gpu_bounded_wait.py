"""The bounded waits of the staging kernels end a launch with an error
status instead of hanging: a test hook stops the fluid-only kernel's copy
warp from issuing the first tile's copies, so every CTA's wait for its tile
runs out (after a limit of 2 ms set through the wait-limit flag), the kernel
returns, and the next synchronising call reports MCLBM_ERR_TIMEOUT.  No GPU
fault is involved: the copies are simply never issued.  Afterwards the
context is usable and a re-initialised lattice steps exactly like a fresh
one."""
import time

import numpy as np
import pytest

from paper_2111_08666_gb300 import media, mclbm

pytestmark = pytest.mark.gpu


def test_unstaged_tile_wait_runs_out_and_reports_timeout():
    m = media.make_disk_medium(160, 64, 4, radius="uniform", r_lo=3.0, r_hi=6.0, porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.3)
    rho1, rho2 = media.drainage_densities(m.solid)
    kw = dict(prec="fp32", kernel=4, nu1=(1.7 - 0.5) / 3, nu2=(0.62 - 0.5) / 3, rho_in1=1.01,
              rho_out2=1.0)
    g = mclbm.Lattice(m.solid, xi, **kw)
    g.init(rho1, rho2)
    g.step(5)
    g.sync()
    mclbm.mclbm_set_flag(g.h, mclbm.MCLBM_FLAG_WAIT_LIMIT_US, 2000)
    mclbm.mclbm_set_flag(g.h, mclbm.MCLBM_FLAG_TEST_NO_COPY, 1)
    t0 = time.perf_counter()
    g.step(1)
    with pytest.raises(mclbm.MclbmError) as e:
        g.sync()
    assert e.value.code == mclbm.MCLBM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0      # the kernel gave up and returned
    g.sync()                                     # the status is reported once
    # the hook off, the lattice re-initialised: the same trajectory as a fresh one
    mclbm.mclbm_set_flag(g.h, mclbm.MCLBM_FLAG_TEST_NO_COPY, 0)
    g.init(rho1, rho2)
    g.step(20)
    h = mclbm.Lattice(m.solid, xi, **kw)
    h.init(rho1, rho2)
    h.step(20)
    assert np.array_equal(g.populations(), h.populations())


def test_wait_limit_flag_bounds():
    solid = np.zeros((8, 8), np.uint8)
    g = mclbm.Lattice(solid, prec="fp32", periodic_y=True)
    for bad in (0, -5, 10_000_001):
        with pytest.raises(mclbm.MclbmError) as e:
            mclbm.mclbm_set_flag(g.h, mclbm.MCLBM_FLAG_WAIT_LIMIT_US, bad)
        assert e.value.code == mclbm.MCLBM_ERR_ARG
    mclbm.mclbm_set_flag(g.h, mclbm.MCLBM_FLAG_WAIT_LIMIT_US, 1)
