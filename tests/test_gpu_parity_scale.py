"""Parity with the FP64 oracle at sizes where the persistent step kernels
walk many tiles per CTA (next-tile prefetch, table and record double
buffers, the tile loop), and of every case of the 24-lattice batch.

Workload: the 1024x512 heterogeneous lognormal disk medium of seed 1
(porosity 0.6, water-wet theta = 50 deg, viscosity ratio 10) under driven
primary drainage, rho_in1 = 1.005 and rho_out2 = 1 (Set-3).  The fluid-only kernel cuts
the lattice into 1460 tiles (12-row bands, at most 256 fluid nodes each)
and walks about 3.2 of them per CTA with 456 resident CTAs, the dense tile
kernel about 3.4 tiles of 32 x 16 per CTA.

The oracle runs once per module: the densities and diagnostics after 200,
1000, 2000, ..., 10000 steps.

Bars (FP32 storage and arithmetic against FP64): densities within 1e-4
of each component's own scale (the largest density of that component),
saturations within 1e-3 absolute."""
import numpy as np
import pytest

import oracle
from paper_2111_08666_gb300 import media, mclbm

pytestmark = pytest.mark.gpu

CHECKS = (200, 1000, 2000, 4000, 6000, 8000, 10000)


def _workload():
    c = media.config_paper_scale(1024, 512, 1)
    kw = dict(nu1=c["nu1"], nu2=c["nu2"], rho_in1=1.005, rho_out2=1.0)
    return c, kw


@pytest.fixture(scope="module")
def oracle_run():
    c, kw = _workload()
    o = oracle.Oracle(c["solid"], c["xi"], **kw)
    o.init(c["rho1"], c["rho2"])
    snaps = {}
    done = 0
    for s in CHECKS:
        o.step(s - done)
        done = s
        snaps[s] = (o.density().copy(), o.diagnostics())
    return snaps


def density_errors(got, want):
    """Per component: max |rho_gpu - rho_oracle| / max rho_oracle."""
    return [float(np.max(np.abs(got[k] - want[k])) / np.max(want[k])) for k in range(2)]


@pytest.mark.parametrize("kernel", [3, 4])
def test_fp32_kernels_match_oracle_paper_scale_200_steps(oracle_run, kernel):
    """The default fluid-only step (kernel 4) and the dense TMA tile step
    (kernel 3) against the oracle after 200 driven steps."""
    c, kw = _workload()
    g = mclbm.Lattice(c["solid"], c["xi"], prec="fp32", kernel=kernel, **kw)
    g.init(c["rho1"], c["rho2"])
    g.step(200)
    want, dw = oracle_run[200]
    errs = density_errors(g.density(), want)
    print(f"kernel {kernel}: density errors after 200 steps {errs}")
    assert max(errs) < 1e-5
    dg = g.diagnostics()
    assert abs(dg["sw_mass"] - dw["sw_mass"]) < 1e-6
    assert abs(dg["sw_count"] - dw["sw_count"]) <= 2.0 / dw["n_fluid"]
    assert dg["n_fluid"] == dw["n_fluid"]


def test_fp32_paper_scale_1e4_steps(oracle_run):
    """The FP32 bar of the paper-scale workload: densities and saturations
    after 10^4 driven steps, recorded every 1000-2000 steps (the curve the
    design notes report)."""
    c, kw = _workload()
    g = mclbm.Lattice(c["solid"], c["xi"], prec="fp32", **kw)
    g.init(c["rho1"], c["rho2"])
    done = 0
    rows = []
    for s in CHECKS:
        g.step(s - done)
        done = s
        want, dw = oracle_run[s]
        dg = g.diagnostics()
        errs = density_errors(g.density(), want)
        rows.append((s, errs[0], errs[1], abs(dg["sw_mass"] - dw["sw_mass"]),
                     abs(dg["sw_count"] - dw["sw_count"]), dw["sw_mass"]))
    for r in rows:
        print("steps %5d  density err %.2e %.2e  dSw mass %.2e count %.2e  (Sw %.5f)" % r)
    for s, e1, e2, dsm, dsc, _ in rows:
        assert dsm <= 1e-3 and dsc <= 1e-3, s
        assert max(e1, e2) < 1e-4, s


def test_every_batch_case_matches_the_oracle():
    """The 24-case batched workload (lattices 256x256 to 1024x512, seeds
    10-33, theta 30-150 deg, M = 1, 10, 50; FP32) advanced by the batched
    persistent launch under its graph; every case against the oracle after
    64 + 37 steps (tuner steps, graph replays and a remainder)."""
    cases = [media.config_batch(k) for k in range(24)]
    p = mclbm.PRECISIONS["fp32"]
    b = mclbm.mclbm_batch_create(cases, p)
    steps = 16 * 6 + 5
    try:
        mclbm.mclbm_batch_step(b, steps)
        info = mclbm.mclbm_batch_info(b)
        assert info["steps"] == steps and info["cases"] == 24
        worst = []
        for k, c in enumerate(cases):
            ny, nx = c["solid"].shape
            view = mclbm.LatticeView(b, k, ny, nx, p)
            o = oracle.Oracle(c["solid"], c["xi"], nu1=c["nu1"], nu2=c["nu2"],
                              rho_in1=c["rho_in1"], rho_out2=c["rho_out2"])
            o.init(c["rho1"], c["rho2"])
            o.step(steps)
            errs = density_errors(view.density(), o.density())
            worst.append(max(errs))
            dg, do = view.diagnostics(), o.diagnostics()
            assert dg["n_fluid"] == do["n_fluid"]
            assert abs(dg["sw_mass"] - do["sw_mass"]) < 1e-6, k
        print("batch cases, worst density error per case:", ["%.1e" % e for e in worst])
        assert max(worst) < 1e-5
    finally:
        mclbm.mclbm_batch_destroy(b)
