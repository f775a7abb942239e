"""Batched persistent stepping: every case of a batch computes what the same
lattice computes alone, whatever kernel, tile shape and grid the tuner
picks and across graph replays.  The tuner's candidates include the tile
kernel and the fluid-only kernel, which differ in how the compiler fuses
FP32 multiply-adds, so the comparison is to rounding (the bounds of the
kernel-agreement test)."""
import numpy as np
import pytest

from paper_2111_08666_gb300 import media, mclbm

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    specs = [(96, 48, 0, -0.4, (1.7, 0.62), True), (75, 41, 1, 0.2, (1.0, 1.0), False),
             (130, 70, 2, -0.55, (3.5, 0.62), True), (64, 64, 3, 0.5, (0.62, 0.62), False)]
    for nx, ny, seed, xi, (t1, t2), drained in specs:
        m = media.make_disk_medium(nx, ny, seed, radius="uniform", r_lo=3.0, r_hi=6.0,
                                   porosity=0.72, reservoir=6)
        if drained:
            r1, r2 = media.drainage_densities(m.solid)
            bc = dict(rho_in1=1.01, rho_out2=1.0)
        else:
            r1, r2 = media.droplet_densities(nx, ny, nx / 3, ny / 2, 6, solid=m.solid)
            bc = dict(rho_in1=-1.0, rho_out2=-1.0)
        out.append(dict(solid=m.solid, xi=media.uniform_xi(m.solid, xi), rho1=r1, rho2=r2,
                        nu1=(t1 - 0.5) / 3, nu2=(t2 - 0.5) / 3, **bc))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp16dev"])
def test_batch_matches_single_lattices(prec):
    cases = _cases()
    p = mclbm.PRECISIONS[prec]
    b = mclbm.mclbm_batch_create(cases, p)
    try:
        steps = 16 * 4 + 7    # tuner steps, graph replays and a remainder
        mclbm.mclbm_batch_step(b, steps)
        info = mclbm.mclbm_batch_info(b)
        assert info["steps"] == steps and info["cases"] == 4 and info["graph"] == 1
        assert info["shape"] in (0, 1, 2, 3)
        for k, c in enumerate(cases):
            ny, nx = c["solid"].shape
            view = mclbm.LatticeView(b, k, ny, nx, p)
            alone = mclbm.Lattice(c["solid"], c["xi"], prec=p, nu1=c["nu1"], nu2=c["nu2"],
                                  rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], kernel=3)
            alone.init(c["rho1"], c["rho2"])
            alone.step(steps)
            fa, fb = alone.populations(), view.populations()
            tol = {"fp32": 4e-6, "fp16dev": 1e-3}[prec]
            assert np.max(np.abs(fa - fb)) <= tol * np.max(np.abs(fa)), (k, np.max(np.abs(fa - fb)))
            da, db = alone.diagnostics(), view.diagnostics()
            assert da["mass1"] == pytest.approx(db["mass1"], rel=tol)
        # a parameter change through a view is picked up (graph re-captured)
        view0 = mclbm.LatticeView(b, 0, *cases[0]["solid"].shape, p)
        view0.set_pressure_bc(1.02, 1.0)
        mclbm.mclbm_batch_step(b, 40)
        assert mclbm.mclbm_batch_info(b)["steps"] == steps + 40
    finally:
        mclbm.mclbm_batch_destroy(b)


def test_batch_rejects_fp64_and_too_many_cases():
    c = _cases()[:1]
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_batch_create(c, mclbm.MCLBM_FP64)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_batch_create(c * 33, mclbm.MCLBM_FP32)


def test_batch_cases_keep_their_own_collision_and_boundary_treatment():
    """Per-case parameters set through views: one case on the MRT variant,
    one on Set-1, one on Set-2, one unchanged; each matches the same lattice
    stepped alone with the same settings."""
    cases = _cases()
    p = mclbm.PRECISIONS["fp32"]
    settings = [dict(mrt=True, s_e=1.1, s_eps=1.2, s_q=1.5), dict(bc_set=1, rho_in2=0.03, rho_out1=0.025),
                dict(bc_set=2), dict()]
    b = mclbm.mclbm_batch_create(cases, p)
    try:
        views = [mclbm.LatticeView(b, k, *c["solid"].shape, p) for k, c in enumerate(cases)]
        for v, st in zip(views, settings):
            if "mrt" in st:
                v.set_mrt(True, st["s_e"], st["s_eps"], st["s_q"])
            if "bc_set" in st:  # the Eq. 26/27 records were taken when the batch was created
                v.set_bc(st["bc_set"], st.get("rho_in2", 0.0), st.get("rho_out1", 0.0))
        steps = 16 * 3 + 5
        mclbm.mclbm_batch_step(b, steps)
        for k, (c, st) in enumerate(zip(cases, settings)):
            alone = mclbm.Lattice(c["solid"], c["xi"], prec=p, nu1=c["nu1"], nu2=c["nu2"],
                                  rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], kernel=3, **st)
            alone.init(c["rho1"], c["rho2"])
            alone.step(steps)
            fa, fb = alone.populations(), views[k].populations()
            assert np.max(np.abs(fa - fb)) <= 4e-6 * np.max(np.abs(fa)), (k, np.max(np.abs(fa - fb)))
    finally:
        mclbm.mclbm_batch_destroy(b)
