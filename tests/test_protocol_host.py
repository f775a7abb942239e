"""Host logic of the quasi-static protocol drivers, no GPU (Sec. 4.2): the
pressure schedules of the hysteresis sweep and of the precision report, the
per-level bookkeeping of a swept case (a level ends when S_w by mass changed
by less than the tolerance over one window, when it reaches the step cap, or
when S_w is no longer finite), and the end points read from a curve: the
threshold capillary pressure (the first drainage level whose water
saturation by count falls below 0.95), the irreducible water (the last
drainage level) and the residual oil (one minus the highest water
saturation of forced imbibition).  A scripted stand-in for a lattice view
replaces the GPU."""
import math

import pytest

from paper_2111_08666_gb300 import hysteresis, precision, trapped


class FakeView:
    """Returns scripted diagnostics, one per call; records the boundary
    densities it is given."""

    def __init__(self, sw_seq, pc=0.001):
        self.sw_seq = list(sw_seq)
        self.i = 0
        self.bc = []
        self.pc = pc

    def set_pressure_bc(self, r_in, r_out):
        self.bc.append((r_in, r_out))

    def diagnostics(self):
        sw = self.sw_seq[min(self.i, len(self.sw_seq) - 1)]
        self.i += 1
        return dict(sw_mass=sw, sw_count=sw, pc=self.pc, p_in=0.34, p_out=0.33)


def test_hysteresis_schedule_endpoints():
    lv = hysteresis.schedule(0.002, 5, 4, 0.01, 3)
    phases = [p for _, _, p in lv]
    assert phases == ["drainage"] * 6 + ["spontaneous"] * 4 + ["forced"] * 3
    assert lv[0] == (1.0, 1.0, "drainage")
    assert lv[5][0] == pytest.approx(1.01) and lv[5][1] == 1.0
    # spontaneous imbibition lowers the inlet back to 1 in equal steps
    assert [r for r, _, _ in lv[6:10]] == pytest.approx([1.0075, 1.005, 1.0025, 1.0])
    # forced imbibition raises the outlet density of component 2
    assert [(r_in, r_out) for r_in, r_out, _ in lv[10:]] == pytest.approx(
        [(1.0, 1.01), (1.0, 1.02), (1.0, 1.03)])


def test_run_ends_a_level_on_convergence_cap_or_non_finite():
    levels = [(1.0, 1.0, "drainage"), (1.01, 1.0, "drainage"), (1.02, 1.0, "drainage")]
    # level 1: start 0.9, then changes of 1e-3, 1e-7 (converged after 2 windows);
    # level 2: start, then changes above tol until the cap of 3 windows;
    # level 3: start, then NaN
    sw = [0.9, 0.899, 0.8989999,            # level 1 (initial read, two checks)
          0.8989999, 0.88, 0.87, 0.86,      # level 2 (initial read, three checks, capped)
          0.86, float("nan")]               # level 3 (initial read, one check)
    v = FakeView(sw)
    run = hysteresis.Run(v, theta=50.0, xi=-0.4, levels=levels, window=1000, tol=1e-6,
                         max_steps=3000)
    while not run.done:
        run.check()
    assert v.bc == [(1.0, 1.0), (1.01, 1.0), (1.02, 1.0)]
    p = run.points
    assert [q["steps"] for q in p] == [2000, 3000, 1000]
    assert [q["converged"] for q in p] == [True, False, False]
    assert p[0]["sw_mass"] == pytest.approx(0.8989999)
    assert p[1]["sw_mass"] == pytest.approx(0.86)
    assert math.isnan(p[2]["sw_mass"])


def _points(drain, spont, forced):
    pts = [dict(phase="drainage", pc=0.001 * (k + 1), sw_count=s, steps=1000, converged=True)
           for k, s in enumerate(drain)]
    pts += [dict(phase="spontaneous", pc=0.0, sw_count=s, steps=1000, converged=True) for s in spont]
    pts += [dict(phase="forced", pc=-0.001, sw_count=s, steps=1000, converged=k != 1)
            for k, s in enumerate(forced)]
    return pts


def test_summary_end_points():
    run = hysteresis.Run.__new__(hysteresis.Run)
    run.theta, run.xi = 22.0, -0.55
    run.points = _points(drain=[1.0, 0.97, 0.94, 0.6, 0.45], spont=[0.5, 0.7],
                         forced=[0.75, 0.81, 0.58])
    s = hysteresis.summarize(run)
    # threshold: the first drainage level below S_w = 0.95 (the third, pc 0.003)
    assert s["pc_threshold"] == pytest.approx(0.003)
    assert s["sw_irreducible"] == pytest.approx(0.45)
    assert s["sw_at_pc0"] == pytest.approx(0.7)
    # residual oil at the highest forced-imbibition saturation, not the last
    assert s["so_residual"] == pytest.approx(1.0 - 0.81)
    assert s["sw_forced_last"] == pytest.approx(0.58)
    assert s["levels"] == 10 and s["unconverged"] == 1 and s["steps"] == 10000


def test_summary_without_a_threshold():
    run = hysteresis.Run.__new__(hysteresis.Run)
    run.theta, run.xi = 110.0, 0.2
    run.points = _points(drain=[0.99, 0.98], spont=[0.985], forced=[0.99])
    assert hysteresis.summarize(run)["pc_threshold"] is None


def test_precision_schedule_and_residuals():
    lv = precision.schedule()
    assert len(lv) == 20
    assert [p for _, _, p in lv] == ["drainage"] * 10 + ["spontaneous"] * 5 + ["forced"] * 5
    assert lv[9][0] == pytest.approx(1.02) and lv[14][0] == pytest.approx(1.0)
    assert lv[-1][:2] == pytest.approx((1.0, 1.02)) and lv[-1][2] == "forced"
    levels = [precision.Level(r_in, r_out, ph, 0.0, 0.9 - 0.01 * k, 0.0, 1.0, 1.0)
              for k, (r_in, r_out, ph) in enumerate(lv)]
    sw_i, so_r = precision.residual_saturations(levels)
    assert sw_i == pytest.approx(0.9 - 0.09)        # the tenth level, the last drainage one
    assert so_r == pytest.approx(1.0 - (0.9 - 0.19))  # one minus the last level's S_w


def test_trapped_summary_takes_the_record_nearest_mid():
    recs = [dict(step=s, sw_mass=0.1, cavity_water=100 - s // 100, front_water=50, behind_water=40 - s // 250,
                 water=200 - s // 50) for s in (0, 400, 1000, 1600)]
    out = trapped.summarize(dict(bc_set=3, steps=1600, seconds=1.0, records=recs), t_mid=900)
    assert out["t_mid"] == 1000
    assert out["cavity_water"] == [100, 90, 84]
    assert out["cavity_water_change"] == pytest.approx((84 - 90) / 90)
    assert out["front_water_change"] == 0.0
    assert out["water"] == [200, 180, 168]
