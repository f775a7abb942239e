"""Storage-precision protocol: drainage then imbibition on the 128x64 disk
medium, the same fixed schedule for every storage precision, so that the
(P_c, S_w) points of the variants correspond one to one.

Schedule (2 x 10^5 steps with the default 10^4 steps per level):
  drainage     rho_in1 = 1.002, 1.004, ..., 1.020   (rho_out2 = 1)
  spontaneous  rho_in1 = 1.016, 1.012, 1.008, 1.004, 1.000
  forced       rho_out2 = 1.004, 1.008, ..., 1.020  (rho_in1 = 1)
(Sec. 4.2.1-4.2.2: the inlet density of the non-wetting component raised
level by level, then lowered, then the outlet density of the wetting one
raised.)  Each level runs a fixed number of steps rather than to a
saturation tolerance, so that no variant stops earlier than another.

A closed box (the same geometry with periodic x, no open boundary) gives
the per-component mass drift, which is exactly zero for the method.

The functions only call ``set_pressure_bc``, ``step`` and ``diagnostics`` of
the lattice object they are given; every step runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass


def schedule():
    """(rho_in1, rho_out2, phase) of the 20 levels."""
    lv = [(1.0 + 0.002 * k, 1.0, "drainage") for k in range(1, 11)]
    lv += [(1.02 - 0.004 * k, 1.0, "spontaneous") for k in range(1, 6)]
    lv += [(1.0, 1.0 + 0.004 * k, "forced") for k in range(1, 6)]
    return lv


@dataclass
class Level:
    rho_in1: float
    rho_out2: float
    phase: str
    pc: float
    sw_mass: float
    sw_count: float
    mass1: float
    mass2: float


def run_protocol(lat, steps_per_level: int = 10000) -> list[Level]:
    """Advance ``lat`` through the schedule; one record per level."""
    out = []
    for r_in, r_out, phase in schedule():
        lat.set_pressure_bc(r_in, r_out)
        lat.step(steps_per_level)
        d = lat.diagnostics()
        out.append(Level(r_in, r_out, phase, d["pc"], d["sw_mass"], d["sw_count"], d["mass1"],
                         d["mass2"]))
    return out


def residual_saturations(levels: list[Level]) -> tuple[float, float]:
    """(S_w at the end of drainage, 1 - S_w at the end of forced imbibition),
    by mass: the irreducible water and residual oil of the schedule."""
    last_drain = [lv for lv in levels if lv.phase == "drainage"][-1]
    return last_drain.sw_mass, 1.0 - levels[-1].sw_mass


def closed_box_drift(lat, steps: int) -> tuple[float, float]:
    """Relative change of each component's mass over ``steps`` steps of a
    lattice without open boundaries."""
    d0 = lat.diagnostics()
    lat.step(steps)
    d1 = lat.diagnostics()
    return d1["mass1"] / d0["mass1"] - 1.0, d1["mass2"] / d0["mass2"] - 1.0
