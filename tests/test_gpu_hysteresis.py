"""The drainage/imbibition driver of Sec. 4.2 (wettability states on the
block stand-in, advanced together as the cases of one batch) runs through
the C ABI and records one converged-or-capped (P_c, S_w) point per
pressure level for every case."""
import pytest

from paper_2111_08666_gb300 import hysteresis

pytestmark = pytest.mark.gpu


def test_hysteresis_sweep_levels_and_summary():
    levels = hysteresis.schedule(0.01, 3, 2, 0.01, 2)
    assert [lv[2] for lv in levels] == ["drainage"] * 4 + ["spontaneous"] * 2 + ["forced"] * 2
    runs, steps, _ = hysteresis.sweep([22.0, 110.0], levels, window=500, tol=1e-6, max_steps=3000)
    assert steps <= len(levels) * 3000 and steps % 500 == 0
    for r in runs:
        assert len(r.points) == len(levels)
        assert all(p["steps"] <= 3000 and p["steps"] % 500 == 0 for p in r.points)
        dr = [p for p in r.points if p["phase"] == "drainage"]
        # raising the inlet density raises the capillary pressure
        assert dr[-1]["pc"] > dr[0]["pc"]
        s = hysteresis.summarize(r)
        assert 0.0 <= s["sw_irreducible"] <= 1.0 and 0.0 <= s["so_residual"] <= 1.0
    # the oil-wet medium drains further at the same pressures
    assert runs[1].points[3]["sw_count"] < runs[0].points[3]["sw_count"]


def test_batched_sweep_matches_lattices_stepped_alone():
    """A case of the batched sweep follows the same levels as the same
    wettability state stepped as a lattice of its own (FP32, to rounding):
    the step counts of every level agree and the saturations within 1e-4."""
    import numpy as np
    from paper_2111_08666_gb300 import mclbm, media
    levels = hysteresis.schedule(0.01, 2, 1, 0.01, 1)
    runs, _, _ = hysteresis.sweep([50.0], levels, window=500, tol=1e-6, max_steps=2000)
    c = media.config_block_hysteresis(50.0)
    lat = mclbm.Lattice(c["solid"], c["xi"], prec="fp32", nu1=c["nu1"], nu2=c["nu2"], rho_in1=1.0,
                        rho_out2=1.0, kernel=3)
    lat.init(c["rho1"], c["rho2"])
    alone = hysteresis.Run(lat, 50.0, c["xi_value"], levels, 500, 1e-6, 2000)
    while not alone.done:
        lat.step(500)
        alone.check()
    for a, b in zip(runs[0].points, alone.points):
        assert a["rho_in1"] == b["rho_in1"] and a["rho_out2"] == b["rho_out2"]
        assert abs(a["sw_mass"] - b["sw_mass"]) < 1e-4
    lat.close()
    assert np.isfinite([p["pc"] for p in runs[0].points]).all()
