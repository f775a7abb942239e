"""The warm/cold drainage-curve driver of the learned warm start, no GPU
(reading #22: two independent curves from the same relaxed start; the warm
curve blends the network's prediction in only where it predicts at least
``gate`` flipped fluid nodes; a curve whose lattice diverges is recorded and
stopped).  A scripted stand-in replaces the lattice and the network: a
lattice relaxes its saturation halfway to the level's target per window, a
blend puts it on the target at once, and a blend can be scripted to make
the lattice diverge."""
import numpy as np
import pytest

from paper_2111_08666_gb300 import mclbm, warmstart


class FakeLattice:
    created = []
    # creation index -> the blends (1, 2, ...) after which that lattice diverges
    diverge_on_blend = {}

    def __init__(self, solid, xi, prec, nu1, nu2, rho_in1, rho_out2, stream=None):
        self.h = self
        self.solid = np.asarray(solid)
        self.sw = self.target = 0.99
        self.bc = []
        self.diverged = False
        self.blends = 0
        self.closed = False
        self.diverge_on = FakeLattice.diverge_on_blend.get(len(FakeLattice.created), set())
        FakeLattice.created.append(self)

    def init(self, rho1, rho2):
        pass

    def set_pressure_bc(self, r_in, r_out):
        self.bc.append((r_in, r_out))
        self.target = 0.99 - 2.0 * (r_in - 1.0)

    def step(self, n):
        if not self.diverged:
            self.sw += 0.5 * (self.target - self.sw)

    def diagnostics(self):
        return dict(sw_mass=float("nan") if self.diverged else self.sw, pc=0.001)

    def sync(self):
        if self.diverged:
            raise mclbm.MclbmError(mclbm.MCLBM_ERR_DIVERGED, "diverged")

    def phase(self):
        # oil (phase > 0) in the first column, water elsewhere
        p = -np.ones(self.solid.shape, np.float32)
        p[:, 0] = 1.0
        return p

    def close(self):
        self.closed = True


class FakeNet:
    """Predicts the current phase field with n more oil nodes on the level's
    n-th call: the first n water nodes (columns 1.., row by row)."""

    def __init__(self, flips_per_level):
        self.flips = list(flips_per_level)
        self.calls = 0

    def infer(self, x):
        n = self.flips[self.calls]
        self.calls += 1
        ny, nx = x.shape[1], x.shape[2]
        phi = np.where(x[0, :, :, 2] > 0, 1.0, -1.0).astype(np.float32)
        water = [(y, c) for y in range(ny) for c in range(nx) if phi[y, c] < 0]
        for y, c in water[:n]:
            phi[y, c] = 1.0
        return phi[None]


@pytest.fixture
def fakes(monkeypatch):
    FakeLattice.created = []
    FakeLattice.diverge_on_blend = {}
    monkeypatch.setattr(mclbm, "Lattice", FakeLattice)
    monkeypatch.setattr(mclbm, "mclbm_set_flag", lambda h, flag, value: None)

    def blend(h, phi, flip):
        h.blends += 1
        if h.blends in h.diverge_on:
            h.diverged = True
        else:
            h.sw = h.target
        # the nodes whose predicted phase has the other sign
        return int(((np.asarray(phi) > 0) != (h.phase() > 0)).sum())

    monkeypatch.setattr(mclbm, "mclbm_blend_phase", blend)
    return FakeLattice


def _case(ny=6, nx=10):
    solid = np.zeros((ny, nx), np.uint8)
    return dict(solid=solid, xi=np.zeros((ny, nx), np.float32), nu1=0.4, nu2=0.04, rho_in1=1.0,
                rho_out2=1.0, rho1=np.ones((ny, nx)), rho2=np.ones((ny, nx)))


def test_gate_blend_and_divergence_bookkeeping(fakes):
    net = FakeNet([12, 3, 5, 12])
    # the warm lattice (created second) diverges on its third blend (level 4)
    fakes.diverge_on_blend = {1: {3}}
    recs = warmstart.drainage_curves(net, _case(), levels=4, d_rho=0.005, window=1000, tol=1e-6,
                                     max_steps=40000, flip=0.0, gate=5)
    cold, warm = FakeLattice.created
    assert len(recs) == 4
    # both curves get each level's inlet density (rho_in = 1 + level * d_rho)
    assert [r for r, _ in cold.bc] == pytest.approx([1.005, 1.01, 1.015, 1.02])
    assert [r for r, _ in warm.bc] == pytest.approx([1.005, 1.01, 1.015, 1.02])
    r1, r2, r3, r4 = recs
    # level 1: 12 predicted flips >= gate: blended, on target after one window
    assert r1["nodes_predicted"] == 12 and r1["nodes_changed"] == 12
    assert r1["converged_warm"] and r1["steps_warm"] == 1000
    # the cold curve halves its distance per window: 0.01 / 2^k < 1e-6 at k = 14
    assert r1["converged_cold"] and r1["steps_cold"] == 14000
    assert r1["sw_cold"] == pytest.approx(r1["sw_warm"], abs=1e-5)
    # level 2: 3 predicted flips < gate: no blend, the warm curve relaxes like the cold one
    assert r2["nodes_predicted"] == 3 and r2["nodes_changed"] == 0
    assert r2["steps_warm"] == r2["steps_cold"]
    # level 3: exactly gate predicted flips: blended
    assert r3["nodes_predicted"] == 5 and r3["nodes_changed"] == 5 and r3["steps_warm"] == 1000
    # level 4: the blend makes the warm lattice diverge; it is recorded, closed and stopped
    assert r4["diverged_warm"] and r4["steps_warm"] is None and np.isnan(r4["sw_warm"])
    assert "pc_warm" not in r4 and warm.closed
    assert not r4["diverged_cold"] and r4["converged_cold"] and "pc_cold" in r4
    # the warm wall time of a level counts the prediction and the blend
    assert r1["sec_warm"] >= r1["sec_predict"] > 0.0
