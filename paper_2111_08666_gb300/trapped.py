"""Trapped volume under the three inlet/outlet treatments (Sec. 4.1): the
invading component 1 flows past a U-shaped wall whose cup, open towards the
inlet, holds water (component 2) and a droplet of component 1; Sec. 2.3
reports that Set-1 and Set-2 let trapped volumes change considerably while
Set-3 keeps them.  This driver runs the same channel under each set on the
GPU and records, every ``every`` steps, the water (nodes with rho2 > rho1,
and the component-2 mass) inside the cup, before its mouth and behind its
closed side, the water in the whole channel and the saturation.  All arithmetic runs in
the CUDA library.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import mclbm, media

SET1_MINOR = 0.027  # Set-1: the other component's fixed density at each end (minority density)


def run_set(case: dict, bc_set: int, steps: int, every: int, prec: str = "fp32",
            snapshots: tuple = ()) -> dict:
    kw = dict(bc_set=bc_set)
    if bc_set == 1:
        kw.update(rho_in2=SET1_MINOR, rho_out1=SET1_MINOR)
    lat = mclbm.Lattice(case["solid"], case["xi"], prec=prec, nu1=case["nu1"], nu2=case["nu2"],
                        rho_in1=case["rho_in1"], rho_out2=case["rho_out2"], **kw)
    lat.init(case["rho1"], case["rho2"])
    fluid = case["solid"] == 0
    regions = {k: case[k] & fluid for k in ("cavity", "front", "behind")}
    rec, snaps = [], {}
    t0 = time.perf_counter()
    n = 0
    while True:
        rho = lat.density()
        water = rho[1] > rho[0]
        r = dict(step=n, water=int((water & fluid).sum()),
                 sw_mass=float(rho[1][fluid].sum() / (rho[0][fluid].sum() + rho[1][fluid].sum())))
        for k, m in regions.items():
            r[f"{k}_water"] = int((water & m).sum())
            r[f"{k}_mass2"] = float(rho[1][m].sum())
        rec.append(r)
        if n in snapshots:
            snaps[n] = (rho[0] - rho[1]).astype(np.float32)
        if n >= steps:
            break
        lat.step(every)
        n += every
    sec = time.perf_counter() - t0
    lat.close()
    return dict(bc_set=bc_set, steps=steps, seconds=sec, records=rec, snapshots=snaps)


def summarize(res: dict, t_mid: int) -> dict:
    """Water nodes in each region at the start, at t_mid (after the
    invasion has passed the U) and at the end, and the relative change of
    each region's water from t_mid to the end."""
    r = res["records"]
    mid = min(r, key=lambda x: abs(x["step"] - t_mid))
    out = dict(bc_set=res["bc_set"], steps=res["steps"], seconds=res["seconds"], t_mid=mid["step"],
               sw_mass_end=r[-1]["sw_mass"])
    for k in ("cavity", "front", "behind", "water"):
        key = k if k == "water" else f"{k}_water"
        a, b = mid[key], r[-1][key]
        out[key] = [r[0][key], a, b]
        out[f"{key}_change"] = (b - a) / a if a else None
    return out


def main(argv=None) -> None:
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=600000)
    ap.add_argument("--every", type=int, default=30000)
    ap.add_argument("--nx", type=int, default=800)
    ap.add_argument("--ny", type=int, default=200)
    ap.add_argument("--sets", type=str, default="1,2,3")
    ap.add_argument("--records", action="store_true", help="print the full time series")
    ap.add_argument("--save", type=str, default="", help="npz file for snapshots of rho1 - rho2")
    a = ap.parse_args(argv)
    case = media.config_u_obstacle(a.nx, a.ny)
    out, arrays = [], {}
    snap_at = (0, a.steps // 4, a.steps // 2, a.steps) if a.save else ()
    for s in [int(v) for v in a.sets.split(",")]:
        res = run_set(case, s, a.steps, a.every, snapshots=snap_at)
        for n, v in res["snapshots"].items():
            arrays[f"set{s}_step{n}"] = v
        summ = summarize(res, a.steps // 4)
        if a.records:
            summ["records"] = res["records"]
        out.append(summ)
        print(json.dumps(summ), flush=True)
    if a.save:
        np.savez_compressed(a.save, solid=case["solid"], cavity=case["cavity"], **arrays)


if __name__ == "__main__":
    main()
