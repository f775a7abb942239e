"""Primary drainage and imbibition at three wettabilities (Sec. 4.2.1-4.2.2):
the capillary-pressure / saturation curves, their hysteresis, the
irreducible water and residual oil saturations.

The wettability states are the cases of one batch (``mclbm_batch_*``): one
persistent launch per step advances all of them, under the batch's CUDA
graph and autotuned step.  Each case follows the quasi-static protocol of
``drainage.py`` on its own: the inlet density of component 1 rises level by
level from equal pressures (drainage), then falls back to the outlet's
(spontaneous imbibition), then the outlet density of component 2 rises
(forced imbibition).  A level ends when S_w by mass changes by less than
``tol`` over ``window`` steps, or after ``max_steps``; a case then moves to
its next level through its batch view while the others continue.  All
arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import json
import math
import time

from . import mclbm, media


def schedule(d_in: float, n_drain: int, n_spont: int, d_out: float, n_forced: int):
    """(rho_in1, rho_out2, phase) of every level."""
    top = 1.0 + d_in * n_drain
    lv = [(1.0 + d_in * k, 1.0, "drainage") for k in range(n_drain + 1)]
    lv += [(top - (top - 1.0) * k / n_spont, 1.0, "spontaneous") for k in range(1, n_spont + 1)]
    lv += [(1.0, 1.0 + d_out * k, "forced") for k in range(1, n_forced + 1)]
    return lv


class Run:
    """One wettability state: a case of the batch, walked through the levels."""

    def __init__(self, view, theta: float, xi: float, levels, window: int, tol: float,
                 max_steps: int):
        self.view, self.theta, self.xi, self.levels = view, theta, xi, levels
        self.window, self.tol, self.max_steps = window, tol, max_steps
        self.k = -1
        self.points = []
        self.next_level()

    def next_level(self):
        self.k += 1
        if self.k < len(self.levels):
            r_in, r_out, _ = self.levels[self.k]
            self.view.set_pressure_bc(r_in, r_out)
            self.steps = 0
            self.prev = self.view.diagnostics()["sw_mass"]

    @property
    def done(self):
        return self.k >= len(self.levels)

    def check(self):
        """After the batch advanced one window: record the level if it has
        converged (or hit the cap) and move on."""
        self.steps += self.window
        d = self.view.diagnostics()
        conv = abs(d["sw_mass"] - self.prev) < self.tol
        if conv or self.steps >= self.max_steps or not math.isfinite(d["sw_mass"]):
            r_in, r_out, phase = self.levels[self.k]
            self.points.append(dict(phase=phase, rho_in1=r_in, rho_out2=r_out, pc=d["pc"],
                                    p_in=d["p_in"], p_out=d["p_out"], sw_count=d["sw_count"],
                                    sw_mass=d["sw_mass"], steps=self.steps, converged=bool(conv)))
            self.next_level()
        else:
            self.prev = d["sw_mass"]


def sweep(thetas, levels, window: int = 1000, tol: float = 1e-6, max_steps: int = 60000,
          stream=None):
    """Run the protocol at every contact angle of ``thetas`` on the block
    stand-in, all cases in one batch.  Returns (runs, batch steps, seconds)."""
    cfgs = [media.config_block_hysteresis(float(t)) for t in thetas]
    cases = [dict(solid=c["solid"], xi=c["xi"], rho1=c["rho1"], rho2=c["rho2"], nu1=c["nu1"],
                  nu2=c["nu2"], rho_in1=1.0, rho_out2=1.0) for c in cfgs]
    b = mclbm.mclbm_batch_create(cases, mclbm.MCLBM_FP32, stream)
    try:
        runs = [Run(mclbm.LatticeView(b, k, c["ny"], c["nx"], mclbm.MCLBM_FP32), c["theta"],
                    c["xi_value"], levels, window, tol, max_steps) for k, c in enumerate(cfgs)]
        t0 = time.perf_counter()
        steps = 0
        while not all(r.done for r in runs):
            mclbm.mclbm_batch_step(b, window)
            steps += window
            for r in runs:
                if not r.done:
                    r.check()
        return runs, steps, time.perf_counter() - t0
    finally:
        mclbm.mclbm_batch_destroy(b)


def summarize(run: Run) -> dict:
    pts = run.points
    dr = [p for p in pts if p["phase"] == "drainage"]
    im = [p for p in pts if p["phase"] != "drainage"]
    # threshold: the first drainage level at which the oil saturation passes
    # 0.05 (the critical oil saturation Sec. 4.2.1 reports is 0.053)
    thr = next((p["pc"] for p in dr if p["sw_count"] < 0.95), None)
    spont_end = [p for p in im if p["phase"] == "spontaneous"]
    forced = [p for p in im if p["phase"] == "forced"]
    # residual oil: at the highest water saturation forced imbibition reaches
    # (a curve that loses water again at higher outlet pressure has passed its
    # residual state); the last level's saturation is reported beside it
    sw_best = max((p["sw_count"] for p in forced), default=im[-1]["sw_count"] if im else None)
    return dict(theta=run.theta, xi=run.xi, pc_threshold=thr, sw_irreducible=dr[-1]["sw_count"],
                sw_at_pc0=spont_end[-1]["sw_count"] if spont_end else None,
                so_residual=1.0 - sw_best if sw_best is not None else None,
                sw_forced_last=forced[-1]["sw_count"] if forced else None,
                levels=len(pts), unconverged=sum(not p["converged"] for p in pts),
                steps=sum(p["steps"] for p in pts))


def main(argv=None) -> None:
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--thetas", type=str, default="22,50,110")
    ap.add_argument("--d-in", type=float, default=0.0015)
    ap.add_argument("--n-drain", type=int, default=30)
    ap.add_argument("--n-spont", type=int, default=12)
    ap.add_argument("--d-out", type=float, default=0.003)
    ap.add_argument("--n-forced", type=int, default=12)
    ap.add_argument("--window", type=int, default=1000)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-steps", type=int, default=60000)
    a = ap.parse_args(argv)
    levels = schedule(a.d_in, a.n_drain, a.n_spont, a.d_out, a.n_forced)
    runs, steps, sec = sweep([float(t) for t in a.thetas.split(",")], levels, a.window, a.tol,
                             a.max_steps)
    for r in runs:
        s = summarize(r)
        s["batch_steps"] = steps
        s["seconds_all"] = sec
        s["points"] = r.points
        print(json.dumps(s), flush=True)


if __name__ == "__main__":
    main()
