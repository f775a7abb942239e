"""Quasi-static capillary-pressure stepping (Sec. 4.2.1 and 4.2.2).

Primary drainage: the outlet density of component 2 stays fixed while the
inlet density of component 1 is raised step by step; after each raise the
lattice is advanced until the water saturation stops changing, and the
converged (P_c, S_w) pair is recorded.  Imbibition reverses the protocol:
the inlet density is lowered until P_c = 0 (spontaneous imbibition), then
the outlet density of component 2 is raised (forced imbibition, negative
P_c).

The driver only calls ``set_pressure_bc``, ``step`` and ``diagnostics`` of
the lattice object it is given, so the same loop runs the CUDA library.
Convergence: |S_w,mass(t) - S_w,mass(t - window)| < tol, checked every
``window`` steps, with S_w by mass (a count changes in steps of one node).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field


@dataclass
class PressureStep:
    rho_in1: float
    rho_out2: float
    pc: float
    p_in: float
    p_out: float
    sw_count: float
    sw_mass: float
    steps: int
    converged: bool
    seconds: float


@dataclass
class Curve:
    points: list[PressureStep] = field(default_factory=list)

    def as_rows(self):
        return [(p.pc, p.sw_count, p.sw_mass, p.steps) for p in self.points]


def relax(lat, *, window: int = 1000, tol: float = 1e-6, max_steps: int = 200_000,
          min_steps: int = 0) -> tuple[int, bool, dict]:
    """Advance until |dS_w| < tol over one window.  Returns (steps, converged,
    diagnostics)."""
    d_prev = lat.diagnostics()
    steps = 0
    while steps < max_steps:
        lat.step(window)
        steps += window
        d = lat.diagnostics()
        if not math.isfinite(d["sw_mass"]):
            return steps, False, d
        if steps >= min_steps and abs(d["sw_mass"] - d_prev["sw_mass"]) < tol:
            return steps, True, d
        d_prev = d
    return steps, False, d_prev


def drainage(lat, rho_in_steps, rho_out2: float = 1.0, *, window: int = 1000,
             tol: float = 1e-6, max_steps: int = 200_000, on_step=None) -> Curve:
    """Primary drainage: for each inlet density, relax and record."""
    curve = Curve()
    for r_in in rho_in_steps:
        lat.set_pressure_bc(float(r_in), float(rho_out2))
        t0 = time.perf_counter()
        if on_step is not None:
            on_step(lat, float(r_in))
        n, ok, d = relax(lat, window=window, tol=tol, max_steps=max_steps)
        curve.points.append(PressureStep(float(r_in), float(rho_out2), d["pc"], d["p_in"],
                                         d["p_out"], d["sw_count"], d["sw_mass"], n, ok,
                                         time.perf_counter() - t0))
    return curve


def imbibition(lat, rho_in_down, rho_out_up, rho_in_floor: float, *, rho_out2: float = 1.0,
               window: int = 1000, tol: float = 1e-6, max_steps: int = 200_000) -> Curve:
    """Imbibition from a drained state: lower the inlet density through
    ``rho_in_down`` (spontaneous part), then hold it at ``rho_in_floor`` and
    raise the outlet density through ``rho_out_up`` (forced part)."""
    curve = Curve()
    for r_in in rho_in_down:
        lat.set_pressure_bc(float(r_in), rho_out2)
        t0 = time.perf_counter()
        n, ok, d = relax(lat, window=window, tol=tol, max_steps=max_steps)
        curve.points.append(PressureStep(float(r_in), rho_out2, d["pc"], d["p_in"], d["p_out"],
                                         d["sw_count"], d["sw_mass"], n, ok,
                                         time.perf_counter() - t0))
    for r_out in rho_out_up:
        lat.set_pressure_bc(float(rho_in_floor), float(r_out))
        t0 = time.perf_counter()
        n, ok, d = relax(lat, window=window, tol=tol, max_steps=max_steps)
        curve.points.append(PressureStep(float(rho_in_floor), float(r_out), d["pc"], d["p_in"],
                                         d["p_out"], d["sw_count"], d["sw_mass"], n, ok,
                                         time.perf_counter() - t0))
    return curve
