"""The drainage/imbibition driver of Sec. 4.2 (three wettabilities on the
block stand-in) runs through the C ABI and records one converged-or-capped
(P_c, S_w) point per pressure level."""
import pytest

from paper_2111_08666_gb300 import hysteresis

pytestmark = pytest.mark.gpu


def test_hysteresis_driver_levels_and_summary():
    levels = hysteresis.schedule(0.01, 3, 2, 0.01, 2)
    assert [lv[2] for lv in levels] == ["drainage"] * 4 + ["spontaneous"] * 2 + ["forced"] * 2
    runs = [hysteresis.Run(t, levels, 500, 1e-6, 3000) for t in (22.0, 110.0)]
    while not all(r.done for r in runs):
        live = [r for r in runs if not r.done]
        for r in live:
            r.advance()
        for r in live:
            r.check()
    for r in runs:
        assert len(r.points) == len(levels)
        assert all(p["steps"] <= 3000 and p["steps"] % 500 == 0 for p in r.points)
        dr = [p for p in r.points if p["phase"] == "drainage"]
        # raising the inlet density raises the capillary pressure
        assert dr[-1]["pc"] > dr[0]["pc"]
        s = hysteresis.summarize(r)
        assert 0.0 <= s["sw_irreducible"] <= 1.0 and 0.0 <= s["so_residual"] <= 1.0
        r.lat.close()
    # the oil-wet medium drains further at the same pressures
    assert runs[1].points[3]["sw_count"] < runs[0].points[3]["sw_count"]
