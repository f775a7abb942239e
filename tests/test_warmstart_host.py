"""Host logic of the warm start: the blended initial densities keep the
previous equilibrium wherever the prediction keeps the phase."""
import numpy as np

from paper_2111_08666_gb300 import warmstart


def test_blend_keeps_unchanged_nodes_and_maps_flipped_ones():
    rng = np.random.default_rng(0)
    ny, nx = 12, 20
    fluid = np.ones((ny, nx), bool)
    fluid[0] = fluid[-1] = False
    rho_prev = np.stack([rng.uniform(0.02, 1.05, (ny, nx)), rng.uniform(0.02, 1.05, (ny, nx))]) * fluid
    phi_prev = np.where(fluid, (rho_prev[0] - rho_prev[1]) / np.maximum(rho_prev.sum(0), 1e-9), 0)
    phi_hat = phi_prev.copy()
    phi_hat[5, 3:9] = -np.sign(phi_prev[5, 3:9]) * 0.8  # six predicted flips
    phi_hat[7, 10] = 1.7                                 # clamped, same sign or flip
    r1, r2, n = warmstart.blend_densities(rho_prev, phi_prev, phi_hat, fluid)
    flipped = fluid & (np.sign(np.clip(phi_hat, -1, 1)) != np.sign(phi_prev))
    assert n == int(flipped.sum()) >= 6
    keep = fluid & ~flipped
    assert np.array_equal(r1[keep], rho_prev[0][keep]) and np.array_equal(r2[keep], rho_prev[1][keep])
    p = np.clip(phi_hat[flipped], -1, 1)
    lo, hi = warmstart.RHO_LO, warmstart.RHO_HI
    assert np.allclose(r1[flipped], lo + (hi - lo) * (1 + p) / 2)
    assert np.allclose(r2[flipped], lo + (hi - lo) * (1 - p) / 2)
    assert not r1[~fluid].any() and not r2[~fluid].any()
