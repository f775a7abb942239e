"""The high-viscosity-ratio driver (SRT of Eq. 1 against the MRT variant) on
a small droplet: both collisions stay finite at M = 1000 with tau2 near
1/2, and the droplet keeps the separated densities of Sec. 3.1 (up to
the compression of a small droplet by its Laplace pressure)."""
import pytest

from paper_2111_08666_gb300 import viscosity_ratio

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_droplet_at_viscosity_ratio_1000(collision):
    r = viscosity_ratio.run(1000.0, collision, steps=4000, n=64)
    assert r["stable"] and r["steps"] == 4000
    assert 0.0 < r["u_max"] < 0.05
    # the radius-8 droplet is compressed by its Laplace pressure (~1.09 inside)
    assert abs(r["rho1_in"] - 1.0) < 0.15 and abs(r["rho1_out"] - 0.027) < 0.005
