"""Learned warm start of the quasi-static drainage protocol (Sec. 4.2): a
U-Net (csrc/unet.cu, BF16 tensor-core kernels) predicts the phase field of
the equilibrium after a pressure step, and the LBM relaxes from it instead
of from the previous equilibrium.

This module holds the host side: the parameter layout and a seeded
initialisation, the network input of a lattice state, and the drivers that
generate training pairs with the batched LBM and compare warm and cold
relaxations.  All arithmetic of the network runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import mclbm

IN_CHANNELS = 8  # input channels of the parameter layout (4 used)
RHO_HI, RHO_LO = 1.0, 0.027  # separated phase densities at G = 3.5 (Sec. 3.1)


def layer_shapes(levels: int, base: int):
    """(name, C_out, C_in, kernel) of every conv, in parameter order."""
    ch = [base << l for l in range(levels)]
    out = []
    for l in range(levels):
        out.append((f"enc{l}a", ch[l], IN_CHANNELS if l == 0 else ch[l - 1], 3))
        out.append((f"enc{l}b", ch[l], ch[l], 3))
    for l in range(levels - 2, -1, -1):
        out.append((f"dec{l}a", ch[l], ch[l] + ch[l + 1], 3))
        out.append((f"dec{l}b", ch[l], ch[l], 3))
    out.append(("head", 1, base, 1))
    return out


def layer_slices(levels: int, base: int):
    """name -> (weight slice, bias slice) of the flat parameter vector."""
    out, o = {}, 0
    for name, co, ci, k in layer_shapes(levels, base):
        n = co * k * k * ci
        out[name] = (slice(o, o + n), slice(o + n, o + n + co))
        o += n + co
    return out


def param_count(levels: int, base: int) -> int:
    return sum(co * k * k * ci + co for _, co, ci, k in layer_shapes(levels, base))


def init_params(levels: int, base: int, seed: int = 0, head_std: float = 0.05) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, a small head."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(param_count(levels, base), np.float32)
    for name, (ws, _bs) in layer_slices(levels, base).items():
        co, ci, k = next((c, i, kk) for n, c, i, kk in layer_shapes(levels, base) if n == name)
        std = head_std if name == "head" else np.sqrt(2.0 / (k * k * ci))
        theta[ws] = rng.normal(0.0, std, ws.stop - ws.start).astype(np.float32)
    return theta


def network_input(solid, xi, phase, dp: float) -> np.ndarray:
    """The 4 input channels [H][W][4]: solid indicator, xi on solid nodes,
    current phase field, pressure step."""
    solid = np.asarray(solid)
    x = np.zeros(solid.shape + (4,), np.float32)
    x[..., 0] = solid != 0
    x[..., 1] = np.where(solid != 0, np.asarray(xi, np.float32), 0.0)
    x[..., 2] = np.where(solid != 0, 0.0, np.asarray(phase, np.float32))
    x[..., 3] = dp
    return x
