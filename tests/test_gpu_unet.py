"""The tensor-core U-Net against the FP64 NumPy reference: forward output,
loss and parameter gradient on the same seeded inputs; the Adam update; a
short training run; the phase-field initialisation of a lattice.

Tolerances follow from the BF16 arithmetic: weights and every activation are
rounded to 8 significant bits (relative error <= 2^-9), about 2 x 2L + 1
roundings on the path to the output, accumulated in FP32.  Random-walk
growth over ~17 roundings gives ~1% relative error on the pre-tanh output,
so the output is compared at 3% (relative L2) and 0.05 (max abs), the loss at
3%, and each layer's gradient by direction (cosine >= 0.99) and norm (10%).
"""
import numpy as np
import pytest

from oracle import unet as ref
from paper_2111_08666_gb300 import mclbm, warmstart

pytestmark = pytest.mark.gpu


def _problem(levels, base, b, h, w, seed):
    theta = warmstart.init_params(levels, base, seed, head_std=0.2)
    rng = np.random.default_rng(seed + 1)
    x4 = rng.normal(0, 1, (b, h, w, 4)).astype(np.float32)
    target = np.tanh(rng.normal(0, 1, (b, h, w))).astype(np.float32)
    mask = (rng.random((b, h, w)) > 0.3).astype(np.float32)
    return theta, x4, target, mask


def _x8(x4):
    x = np.zeros(x4.shape[:3] + (ref.IN_CHANNELS,))
    x[..., :4] = x4
    return x


# widths below 128 take the pixel-gather kernel, multiples of 128 the
# persistent row-tile kernel (512, 256 and 128 over three levels; 1024 to 128
# over four, whose level-2 decoder streams its weights through a two-stage
# ring and expands the upsampled input); a small max_ctas makes each CTA walk
# many tiles, through both accumulator buffers and every stage of its ring
@pytest.mark.parametrize("levels,b,h,w,max_ctas", [(3, 2, 32, 48, 0), (4, 1, 64, 32, 0), (3, 1, 8, 512, 0),
                                                   (3, 1, 8, 512, 3), (4, 1, 8, 1024, 0), (4, 1, 8, 1024, 2)])
def test_forward_matches_reference(levels, b, h, w, max_ctas):
    base = 32
    theta, x4, _, _ = _problem(levels, base, b, h, w, seed=levels)
    assert warmstart.param_count(levels, base) == ref.param_count(levels, base)
    net = mclbm.UNet(levels, base, max_batch=b, max_h=h, max_w=w)
    mclbm.mclbm_unet_set_max_ctas(net.h, max_ctas)
    net.set_params(theta)
    assert np.array_equal(net.params(), theta)
    phi = net.infer(x4)
    want, _ = ref.forward(theta.astype(np.float64), _x8(x4), levels, base)
    err = np.linalg.norm(phi - want) / np.linalg.norm(want)
    assert err < 3e-2, err
    assert np.max(np.abs(phi - want)) < 0.05
    assert np.std(want) > 0.1  # not saturated: the comparison means something
    net.close()


# widths that are multiples of 128 take the shared-tap weight-gradient
# kernel at every level (32 to 256 output channels, in 32-channel slices).
# Its CTAs walk runs of row tiles down 128-pixel strips with the dZ rows in a
# ring: 24 rows with max_ctas 3 make runs long enough to wrap the ring and
# cross strips and images (the rows above and below a tile come from its own
# image); four levels at width 1024 add the 256-channel level; base 64 makes
# a decoder with more (slice, chunk) pairs (8 x 24) than the GPU has SMs, and
# a 512-channel level on the per-tap kernel
@pytest.mark.parametrize("levels,b,h,w,max_ctas,base", [(3, 2, 32, 32, 0, 32), (3, 1, 8, 512, 0, 32),
                                                        (3, 1, 8, 512, 3, 32), (3, 2, 24, 512, 0, 32),
                                                        (3, 2, 24, 512, 3, 32), (4, 1, 8, 1024, 0, 32),
                                                        (4, 1, 8, 1024, 0, 64)])
def test_gradient_matches_reference(levels, b, h, w, max_ctas, base):
    theta, x4, target, mask = _problem(levels, base, b, h, w, seed=7)
    net = mclbm.UNet(levels, base, max_batch=b, max_h=h, max_w=w)
    mclbm.mclbm_unet_set_max_ctas(net.h, max_ctas)
    net.set_params(theta)
    loss, g = net.gradient(x4, target, mask)
    want_loss, want_g, _ = ref.loss_and_gradient(theta.astype(np.float64), _x8(x4),
                                                 target.astype(np.float64),
                                                 mask.astype(np.float64), levels, base)
    assert loss == pytest.approx(want_loss, rel=3e-2)
    for name, (ws, bs) in warmstart.layer_slices(levels, base).items():
        for part, s in (("w", ws), ("b", bs)):
            a, r = g[s].astype(np.float64), want_g[s]
            nr = np.linalg.norm(r)
            if nr < 1e-12:
                continue
            cos = a @ r / (np.linalg.norm(a) * nr)
            assert cos > 0.99, (name, part, cos)
            assert abs(np.linalg.norm(a) / nr - 1) < 0.1, (name, part)
    net.close()


# the shared-tap weight gradient against the per-tap kernel on the same
# network and data: the same BF16 products summed in another order, so they
# agree to FP32 rounding (a wrong dZ row in some ring windows would show as
# a gross difference in the affected taps, which the oracle comparison above,
# loose enough for BF16 error propagation, could let through)
@pytest.mark.parametrize("levels,b,h,w,max_ctas", [(3, 2, 24, 512, 3), (3, 2, 24, 512, 0), (3, 1, 40, 256, 1),
                                                   (4, 1, 16, 1024, 0)])
def test_shared_tap_wgrad_matches_per_tap(levels, b, h, w, max_ctas):
    base = 32
    theta, x4, target, mask = _problem(levels, base, b, h, w, seed=11)
    net = mclbm.UNet(levels, base, max_batch=b, max_h=h, max_w=w)
    mclbm.mclbm_unet_set_max_ctas(net.h, max_ctas)
    net.set_params(theta)
    loss_a, g_shared = net.gradient(x4, target, mask)
    mclbm.mclbm_unet_set_shared_taps(net.h, 0)
    loss_b, g_tap = net.gradient(x4, target, mask)
    assert loss_a == pytest.approx(loss_b, rel=1e-6)  # the forward pass does not use the switch
    for name, (ws, _) in warmstart.layer_slices(levels, base).items():
        a, r = g_shared[ws].astype(np.float64), g_tap[ws].astype(np.float64)
        scale = np.max(np.abs(r))
        assert scale > 0, name
        assert np.max(np.abs(a - r)) <= 1e-3 * scale, (name, np.max(np.abs(a - r)) / scale)
    net.close()


def test_adam_step_follows_its_formula():
    """First Adam step: m = (1 - b1) g, v = (1 - b2) g^2, so the bias-corrected
    update is lr g / (|g| + eps)."""
    levels, base, b, h, w = 2, 32, 1, 16, 16
    theta, x4, target, mask = _problem(levels, base, b, h, w, seed=3)
    net = mclbm.UNet(levels, base, max_batch=b, max_h=h, max_w=w)
    net.set_params(theta)
    _, g = net.gradient(x4, target, mask)
    lr = 1e-3
    net.train_step(x4, target, mask, lr)
    new = net.params()
    big = np.abs(g) > 1e-4
    want = theta - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(new[big], want[big], rtol=0, atol=lr * 1e-3)
    assert np.all(np.abs(new - theta) <= lr * (1 + 1e-3))
    net.close()


def test_training_reduces_the_loss():
    levels, base, b, h, w = 3, 32, 4, 32, 32
    rng = np.random.default_rng(11)
    x4 = rng.normal(0, 1, (b, h, w, 4)).astype(np.float32)
    target = np.tanh(x4[..., 2] + 0.5 * x4[..., 0]).astype(np.float32)
    mask = np.ones((b, h, w), np.float32)
    net = mclbm.UNet(levels, base, max_batch=b, max_h=h, max_w=w)
    net.set_params(warmstart.init_params(levels, base, 5))
    first = net.train_step(x4, target, mask, 2e-3)
    for _ in range(80):
        last = net.train_step(x4, target, mask, 2e-3)
    assert np.isfinite(last) and last < 0.3 * first, (first, last)
    net.close()


def test_init_from_phase_sets_the_densities():
    nx, ny = 40, 20
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    rng = np.random.default_rng(2)
    phi = rng.uniform(-1.2, 1.2, (ny, nx)).astype(np.float32)
    lat = mclbm.Lattice(solid, None, prec="fp64")
    mclbm.mclbm_init_from_phase(lat.h, phi)
    p = np.clip(phi.astype(np.float64), -1, 1)
    fluid = solid == 0
    rho = lat.density()
    for comp, sign in ((1, 1.0), (2, -1.0)):
        want = warmstart.RHO_LO + (warmstart.RHO_HI - warmstart.RHO_LO) * (1 + sign * p) / 2
        got = rho[comp - 1]
        assert np.allclose(got[fluid], want[fluid], rtol=1e-13, atol=0)
    lat.close()
