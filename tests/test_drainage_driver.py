"""The quasi-static P_c stepping loop (Sec. 4.2.1): convergence logic on a
scripted lattice (CPU), and the same loop on the GPU and on the oracle."""
import numpy as np
import pytest

from paper_2111_08666_gb300 import drainage, media


class Scripted:
    """A stand-in lattice whose saturation follows a given sequence."""

    def __init__(self, sw_seq):
        self.sw = list(sw_seq)
        self.k = 0
        self.bc = []
        self.steps = 0

    def set_pressure_bc(self, a, b):
        self.bc.append((a, b))

    def step(self, n):
        self.steps += n
        self.k = min(self.k + 1, len(self.sw) - 1)

    def diagnostics(self):
        s = self.sw[self.k]
        return dict(sw_mass=s, sw_count=s, pc=0.01 * len(self.bc), p_in=0.4, p_out=0.39)


def test_relax_stops_when_saturation_settles():
    lat = Scripted([1.0, 0.9, 0.85, 0.8499, 0.8499, 0.8499])
    n, ok, d = drainage.relax(lat, window=100, tol=1e-3)
    assert ok and n == 300 and d["sw_mass"] == pytest.approx(0.8499)


def test_relax_gives_up_after_max_steps():
    lat = Scripted(np.linspace(1, 0, 50))
    n, ok, _ = drainage.relax(lat, window=10, tol=1e-6, max_steps=100)
    assert not ok and n == 100


def test_drainage_records_one_point_per_pressure_step():
    lat = Scripted([1.0, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5])
    curve = drainage.drainage(lat, [1.001, 1.002, 1.003], window=10, tol=1e-9)
    assert [p.rho_in1 for p in curve.points] == [1.001, 1.002, 1.003]
    assert lat.bc == [(1.001, 1.0), (1.002, 1.0), (1.003, 1.0)]
    assert all(p.converged for p in curve.points)


@pytest.mark.gpu
def test_drainage_curve_gpu_matches_oracle():
    import oracle
    from paper_2111_08666_gb300 import mclbm
    c = media.config_small_fp64()
    xi = media.uniform_xi(c["solid"], -0.4)
    kw = dict(nu1=(1.7 - 0.5) / 3, nu2=(0.62 - 0.5) / 3, rho_in1=1.0, rho_out2=1.0)
    o = oracle.Oracle(c["solid"], xi, **kw)
    o.init(c["rho1"], c["rho2"])
    g = mclbm.Lattice(c["solid"], xi, prec="fp64", **kw)
    g.init(c["rho1"], c["rho2"])
    steps = [1.004, 1.008, 1.012]
    co = drainage.drainage(o, steps, window=200, tol=1e-6, max_steps=1000)
    cg = drainage.drainage(g, steps, window=200, tol=1e-6, max_steps=1000)
    for a, b in zip(cg.points, co.points):
        assert a.steps == b.steps
        assert a.pc == pytest.approx(b.pc, rel=1e-9, abs=1e-12)
        assert a.sw_mass == pytest.approx(b.sw_mass, rel=1e-10)
        assert a.sw_count == b.sw_count
    # drainage: water saturation does not increase as P_c is raised
    sw = [p.sw_mass for p in cg.points]
    assert all(b <= a + 1e-9 for a, b in zip(sw, sw[1:]))


@pytest.mark.gpu
def test_imbibition_curve_gpu_matches_oracle():
    """Imbibition (Sec. 4.2.2) from a drained state, FP64 on the GPU against
    the oracle: the inlet density is lowered (spontaneous part) and then the
    outlet density raised (forced part); every level's step count,
    capillary pressure and saturations agree."""
    import oracle
    from paper_2111_08666_gb300 import mclbm
    c = media.config_small_fp64()
    xi = media.uniform_xi(c["solid"], -0.4)
    kw = dict(nu1=(1.7 - 0.5) / 3, nu2=(0.62 - 0.5) / 3, rho_in1=1.0, rho_out2=1.0)
    o = oracle.Oracle(c["solid"], xi, **kw)
    o.init(c["rho1"], c["rho2"])
    g = mclbm.Lattice(c["solid"], xi, prec="fp64", **kw)
    g.init(c["rho1"], c["rho2"])
    args = dict(window=200, tol=1e-6, max_steps=800)
    for lat in (o, g):
        drainage.drainage(lat, [1.01, 1.02], **args)
    co = drainage.imbibition(o, [1.01, 1.0], [1.01, 1.02], 1.0, **args)
    cg = drainage.imbibition(g, [1.01, 1.0], [1.01, 1.02], 1.0, **args)
    assert len(cg.points) == len(co.points) == 4
    for a, b in zip(cg.points, co.points):
        assert (a.rho_in1, a.rho_out2) == (b.rho_in1, b.rho_out2)
        assert a.steps == b.steps
        assert a.pc == pytest.approx(b.pc, rel=1e-9, abs=1e-12)
        assert a.sw_mass == pytest.approx(b.sw_mass, rel=1e-10)
        assert a.sw_count == b.sw_count
    # the forced part lowers P_c below the spontaneous part's
    assert cg.points[-1].pc < cg.points[1].pc
