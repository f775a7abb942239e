"""The high-viscosity-ratio driver (SRT of Eq. 1 against the MRT variant) on
a small droplet: both collisions stay finite at M = 1000 with tau2 near
1/2, and the FP32 run on the GPU matches the FP64 oracle on the same case
(density fields within the FP32 bar, the spurious-current maximum within
5 %)."""
import numpy as np
import pytest

import oracle
from paper_2111_08666_gb300 import mclbm, media, viscosity_ratio

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_droplet_at_viscosity_ratio_1000(collision):
    r = viscosity_ratio.run(1000.0, collision, steps=4000, n=64)
    assert r["stable"] and r["steps"] == 4000
    assert 0.0 < r["u_max"] < 0.05

    # the same case on the oracle: a radius-8 droplet at rest in a periodic
    # 64 x 64 box, tau1 = 1, nu2 = nu1 / 1000
    n = 64
    solid = np.zeros((n, n), np.uint8)
    rho1, rho2 = media.droplet_densities(n, n, n / 2, n / 2, n / 8)
    kw = dict(nu1=1.0 / 6.0, nu2=1.0 / 6.0 / 1000.0, periodic_y=True,
              **viscosity_ratio.COLLISIONS[collision])
    o = oracle.Oracle(solid, np.zeros((n, n), np.float32), **kw)
    o.init(rho1, rho2)
    o.step(4000)
    g = mclbm.Lattice(solid, None, prec="fp32", **kw)
    g.init(rho1, rho2)
    g.step(4000)
    want, got = o.density(), g.density()
    errs = [float(np.max(np.abs(got[k] - want[k])) / np.max(want[k])) for k in range(2)]
    ux, uy = g.velocity()
    u_gpu = float(np.sqrt(ux * ux + uy * uy).max())
    u_ora = float(np.sqrt(o.ux ** 2 + o.uy ** 2).max())
    print(f"{collision}: density errors {errs}, u_max GPU {u_gpu:.6f} oracle {u_ora:.6f}")
    assert max(errs) < 1e-4
    assert u_gpu == pytest.approx(u_ora, rel=0.05)
    assert r["rho1_in"] == pytest.approx(float(got[0][n // 2, n // 2]), rel=1e-6)
