"""Host logic of the warm start: the network input packs the lattice state
into its four channels (solid indicator, xi on solid nodes, the phase field
on fluid nodes, the pressure step), and the relaxation loop stops on the
saturation tolerance."""
import numpy as np

from paper_2111_08666_gb300 import warmstart


def test_network_input_channels():
    rng = np.random.default_rng(0)
    ny, nx = 12, 20
    solid = (rng.random((ny, nx)) < 0.3).astype(np.uint8)
    xi = np.where(solid != 0, -0.4, 0.7).astype(np.float32)   # a stray xi on fluid is ignored
    phase = rng.uniform(-1, 1, (ny, nx)).astype(np.float32)
    x = warmstart.network_input(solid, xi, phase, 0.5)
    assert x.shape == (ny, nx, 4) and x.dtype == np.float32
    assert np.array_equal(x[..., 0], (solid != 0).astype(np.float32))
    assert np.array_equal(x[..., 1], np.where(solid != 0, np.float32(-0.4), 0).astype(np.float32))
    assert np.array_equal(x[..., 2], np.where(solid != 0, 0, phase).astype(np.float32))
    assert np.all(x[..., 3] == 0.5)


def test_relax_stops_on_tolerance_or_cap():
    seq = iter([1.0, 0.9, 0.8999995, 0.8999990])
    state = {"s": next(seq)}

    def step(n):
        state["s"] = next(seq)
    n, s, ok = warmstart.relax(step, lambda: state["s"], window=10, tol=1e-6, max_steps=100)
    assert ok and n == 20 and s == 0.8999995
    vals = iter(np.linspace(1, 0, 20))
    state["s"] = next(vals)

    def step2(n):
        state["s"] = next(vals)
    n, s, ok = warmstart.relax(step2, lambda: state["s"], window=10, tol=1e-6, max_steps=50)
    assert not ok and n == 50
