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
    # per component, against that component's own scale
    dens_err = max(np.max(np.abs(rho[k] - rho_o[k])) / np.max(np.abs(rho_o[k])) for k in range(2))
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


# --- the precision report: drainage then imbibition, 2 x 10^5 steps ---------------

# variant: (P_c bound, S_w bound) on the largest difference from the FP64
# oracle over the 20 levels of the schedule
REPORT_BOUNDS = {
    "fp64": (1e-10, 1e-10),
    "fp32": (2e-5, 1e-3),
    "fp32dev": (2e-5, 1e-3),
    "fp16dev": (5e-4, 2e-2),
    "bf16dev": (5e-3, 1e-1),
}


@pytest.fixture(scope="module")
def oracle_protocol():
    from paper_2111_08666_gb300 import precision
    c = media.config_small_fp64()
    o = oracle.Oracle(c["solid"], c["xi"], nu1=c["nu1"], nu2=c["nu2"], rho_in1=1.0, rho_out2=1.0)
    o.init(c["rho1"], c["rho2"])
    return precision.run_protocol(o)


@pytest.mark.parametrize("prec", list(REPORT_BOUNDS))
def test_precision_report_drainage_imbibition(oracle_protocol, prec):
    """The 128x64 disk medium (neutral wetting, M = 1) through the fixed
    drainage / spontaneous / forced imbibition schedule of ``precision.py``
    (20 levels of 10^4 steps), each storage precision against the FP64
    oracle: the largest P_c and S_w differences over the levels, the
    residual saturations, and the closed-box mass drift per component over
    2 x 10^5 steps."""
    from paper_2111_08666_gb300 import precision
    c = media.config_small_fp64()
    g = mclbm.Lattice(c["solid"], c["xi"], prec=prec, nu1=c["nu1"], nu2=c["nu2"], rho_in1=1.0,
                      rho_out2=1.0)
    g.init(c["rho1"], c["rho2"])
    got = precision.run_protocol(g)
    want = oracle_protocol
    dpc = max(abs(a.pc - b.pc) for a, b in zip(got, want))
    dsw = max(abs(a.sw_mass - b.sw_mass) for a, b in zip(got, want))
    dswc = max(abs(a.sw_count - b.sw_count) for a, b in zip(got, want))
    swi, sor = precision.residual_saturations(got)
    swi_o, sor_o = precision.residual_saturations(want)
    # closed box: the same geometry and initial state, periodic x
    box = mclbm.Lattice(c["solid"], c["xi"], prec=prec, nu1=c["nu1"], nu2=c["nu2"])
    box.init(c["rho1"], c["rho2"])
    d1, d2 = precision.closed_box_drift(box, 200000)
    print(f"\nPRECISION REPORT {prec}: max |dPc| {dpc:.2e}  max |dSw| mass {dsw:.2e} count {dswc:.2e}  "
          f"S_w,i {swi:.5f} (oracle {swi_o:.5f})  S_o,r {sor:.5f} (oracle {sor_o:.5f})  "
          f"closed-box drift {d1:.2e} {d2:.2e}")
    for a, b in zip(got, want):
        print(f"  {a.phase:12s} rho_in {a.rho_in1:.3f} rho_out {a.rho_out2:.3f}  Pc {a.pc:+.6f} "
              f"({b.pc:+.6f})  Sw {a.sw_mass:.6f} ({b.sw_mass:.6f})")
    bpc, bsw = REPORT_BOUNDS[prec]
    assert dpc < bpc and dsw < bsw
    assert abs(swi - swi_o) < bsw and abs(sor - sor_o) < bsw
