"""Storage-precision variants against the FP64 oracle (precision row of the
hot path): FP32 deviation storage, FP16 and BF16 deviation storage with FP32
arithmetic, FP64 global reductions in all of them.

Each variant runs the 128x64 disk medium (the FP64 workload's geometry) for
10^4 steps with balanced boundary densities, and a closed box for mass
drift.  The printed table is the measured precision report; the asserted
bounds are the ones each variant meets with margin.
"""
import numpy as np
import pytest

import oracle
from paper_2111_08666_gb300 import media, mclbm

pytestmark = pytest.mark.gpu

# variant: (density bound, saturation bound, relative mass drift bound)
BOUNDS = {
    "fp32": (1e-4, 1e-3, 1e-5),
    "fp32dev": (1e-4, 1e-3, 1e-5),
    "fp16dev": (5e-2, 5e-2, 1e-2),
    "bf16dev": (2e-1, 1e-1, 5e-2),
}

_oracle_cache = {}


def _oracle_stable(steps):
    if steps not in _oracle_cache:
        c = media.config_small_fp64()
        o = oracle.Oracle(c["solid"], c["xi"], nu1=c["nu1"], nu2=c["nu2"], rho_in1=1.0,
                          rho_out2=1.0)
        o.init(c["rho1"], c["rho2"])
        o.step(steps)
        _oracle_cache[steps] = (o.density(), o.diagnostics())
    return _oracle_cache[steps]


@pytest.mark.parametrize("prec", list(BOUNDS))
def test_precision_variant_vs_oracle(prec):
    steps = 10000
    rho_o, d_o = _oracle_stable(steps)
    c = media.config_small_fp64()
    g = mclbm.Lattice(c["solid"], c["xi"], prec=prec, nu1=c["nu1"], nu2=c["nu2"],
                      rho_in1=1.0, rho_out2=1.0)
    g.init(c["rho1"], c["rho2"])
    g.step(steps)
    rho = g.density()
    d = g.diagnostics()
    dens_err = np.max(np.abs(rho - rho_o)) / np.max(np.abs(rho_o))
    sw_err = abs(d["sw_mass"] - d_o["sw_mass"])
    swc_err = abs(d["sw_count"] - d_o["sw_count"])

    # closed box (walls, periodic x): per-component mass drift
    nx, ny = 96, 48
    solid = np.zeros((ny, nx), np.uint8)
    solid[:2] = 1
    solid[-2:] = 1
    solid[18:30, 60:72] = 1
    r1, r2 = media.droplet_densities(nx, ny, 30, 20, 10, solid=solid)
    box = mclbm.Lattice(solid, media.uniform_xi(solid, -0.4), prec=prec,
                        nu1=(1.7 - 0.5) / 3, nu2=(0.62 - 0.5) / 3)
    box.init(r1, r2)
    m0 = box.diagnostics()
    box.step(steps)
    m1 = box.diagnostics()
    drift = max(abs(m1["mass1"] / m0["mass1"] - 1), abs(m1["mass2"] / m0["mass2"] - 1))
    print(f"\nPRECISION {prec}: density err {dens_err:.3e}  S_w(mass) err {sw_err:.3e}  "
          f"S_w(count) err {swc_err:.3e}  closed-box mass drift {drift:.3e} after {steps} steps")
    bd, bs, bm = BOUNDS[prec]
    assert np.isfinite(dens_err) and dens_err < bd
    assert sw_err < bs and swc_err < bs
    assert drift < bm
