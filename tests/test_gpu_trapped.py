"""The trapped-volume driver of Sec. 4.1 (three inlet/outlet treatments on
the U-obstacle channel) runs through the C ABI on a small channel and
returns consistent records."""
import numpy as np
import pytest

from paper_2111_08666_gb300 import media, trapped

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc_set", [1, 2, 3])
def test_trapped_volume_driver_small_channel(bc_set):
    case = media.config_u_obstacle(400, 100, arm=6, r_drop=12.0)
    res = trapped.run_set(case, bc_set, steps=4000, every=2000)
    r = res["records"]
    assert [x["step"] for x in r] == [0, 2000, 4000]
    fluid = case["solid"] == 0
    # at step 0 the counts are those of the initial densities
    water0 = (case["rho2"] > case["rho1"]) & fluid
    assert r[0]["water"] == int(water0.sum())
    assert r[0]["cavity_water"] == int((water0 & case["cavity"]).sum())
    for x in r:
        assert 0 <= x["cavity_water"] <= int((case["cavity"] & fluid).sum())
        assert 0.0 < x["sw_mass"] < 1.0 and np.isfinite(x["cavity_mass2"])
    # the invading component advances: the saturation falls
    assert r[-1]["sw_mass"] < r[0]["sw_mass"]
    s = trapped.summarize(res, 2000)
    assert s["cavity_water"][1] == r[1]["cavity_water"]
