"""Pins of the FP64 U-Net reference: central finite differences of the loss
agree with its analytic gradient, and its operations reduce to their
textbook definitions on tiny inputs."""
import numpy as np
import pytest

from oracle import unet


def _problem(levels, base, b=2, h=8, w=8, seed=0):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, unet.param_count(levels, base))
    x = rng.normal(0, 1, (b, h, w, unet.IN_CHANNELS))
    x[..., 4:] = 0.0
    target = np.tanh(rng.normal(0, 1, (b, h, w)))
    mask = (rng.random((b, h, w)) > 0.3).astype(float)
    return theta, x, target, mask


def test_param_layout_counts():
    # 2 levels, 4 channels: enc0a 4*9*8+4, enc0b 4*9*4+4, enc1a 8*9*4+8,
    # enc1b 8*9*8+8, dec0a 4*9*12+4, dec0b 4*9*4+4, head 4+1
    assert unet.param_count(2, 4) == 292 + 148 + 296 + 584 + 436 + 148 + 5


def test_conv3_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 5, 4, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = unet.conv3(x, w, b)
    for (yy, xx, co) in [(0, 0, 0), (2, 1, 1), (4, 3, 0)]:
        s = b[co]
        for ky in range(3):
            for kx in range(3):
                sy, sx = yy + ky - 1, xx + kx - 1
                if 0 <= sy < 5 and 0 <= sx < 4:
                    s += np.dot(x[0, sy, sx], w[co, ky, kx])
        assert y[0, yy, xx, co] == pytest.approx(s, rel=1e-12)


def test_pool_and_upsample_are_adjoint():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(1, 4, 6, 2))
    c = rng.normal(size=(1, 2, 3, 2))
    # <pool(a), c> = <a, pool^T(c)> and <up(c), a> = <c, up^T(a)>
    assert np.sum(unet.pool2(a) * c) == pytest.approx(np.sum(a * unet.pool2_backward(c)))
    assert np.sum(unet.up2(c) * a) == pytest.approx(np.sum(c * unet.up2_backward(a)))


@pytest.mark.parametrize("levels,base", [(2, 4), (3, 2)])
def test_gradient_matches_finite_differences(levels, base):
    theta, x, target, mask = _problem(levels, base)
    loss, grad, _ = unet.loss_and_gradient(theta, x, target, mask, levels, base)
    rng = np.random.default_rng(3)
    idx = rng.choice(theta.size, 40, replace=False)
    eps = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        lp = unet.loss_and_gradient(tp, x, target, mask, levels, base)[0]
        lm = unet.loss_and_gradient(tm, x, target, mask, levels, base)[0]
        fd = (lp - lm) / (2 * eps)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k


# Nearest upsampling followed by a 3x3 convolution, per output phase
# (py, px) = (y mod 2, x mod 2): the fine taps dy of an even output row land
# on coarse rows Y - 1 (dy = -1) and Y (dy = 0, +1); of an odd row on Y
# (dy = -1, 0) and Y + 1 (dy = +1); likewise along x.  Each phase is then a
# 2 x 2 convolution of the coarse input with summed weights: 4 taps instead
# of 9 per output, and no upsampled tensor.  (A reformulation for the
# decoders' upsampled inputs; pinned here against the textbook operations.)
_LAND = {(0, -1): (-1,), (0, 0): (0, 1), (1, 0): (-1, 0), (1, 1): (1,)}
_OFFS = {0: (-1, 0), 1: (0, 1)}


def _phase_kernels(w):
    out = {}
    for py in (0, 1):
        for px in (0, 1):
            out[(py, px)] = {(a, c): sum(w[:, dy + 1, dx + 1, :] for dy in _LAND[(py, a)] for dx in _LAND[(px, c)])
                             for a in _OFFS[py] for c in _OFFS[px]}
    return out


def test_upsample_then_convolve_is_four_coarse_2x2_convolutions():
    rng = np.random.default_rng(5)
    bsz, h, wd, ci, co = 2, 5, 7, 3, 4
    x = rng.normal(size=(bsz, h, wd, ci))
    w = rng.normal(size=(co, 3, 3, ci))
    b = rng.normal(size=co)
    want = unet.conv3(unet.up2(x), w, b)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    got = np.zeros_like(want)
    for (py, px), kern in _phase_kernels(w).items():
        # each phase's four kernels split the nine taps between them
        assert np.allclose(sum(kern.values()), w.sum(axis=(1, 2)))
        acc = np.zeros((bsz, h, wd, co))
        for (a, c), k in kern.items():
            acc += xp[:, 1 + a:1 + a + h, 1 + c:1 + c + wd, :] @ k.T
        got[:, py::2, px::2, :] = acc + b
    assert np.max(np.abs(got - want)) < 1e-12


def test_bf16_round_known_values():
    """Round to nearest, ties to even, at 8 significant bits: exactly
    representable values are kept; a value half an ulp above 1 (ulp 2^-7)
    rounds down to the even 1, three halves up to 1 + 2^-6 ... and signs
    and powers of two are preserved."""
    r = unet.bf16_round
    assert r(1.0) == 1.0 and r(-2.5) == -2.5 and r(0.0) == 0.0
    assert r(1.0 + 2.0 ** -8) == 1.0                 # tie -> even (down)
    assert r(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert r(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert r(3.0 * 2.0 ** -100) == 3.0 * 2.0 ** -100
    x = np.random.default_rng(0).normal(0, 10, 1000)
    rel = np.abs(r(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 and np.all(np.abs(r(r(x)) - r(x)) == 0)


def test_storage_model_is_the_plain_network_without_rounding():
    """store=None and store=identity give the plain FP64 network; the BF16
    model rounds the 3x3 weights only (biases and the head are kept)."""
    levels, base = 2, 8
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 0.3, unet.param_count(levels, base))
    x = rng.normal(0, 1, (1, 8, 8, unet.IN_CHANNELS))
    a, _ = unet.forward(theta, x, levels, base)
    b, _ = unet.forward(theta, x, levels, base, store=lambda v: v)
    assert np.array_equal(a, b)
    q = unet.store_weights(theta, levels, base)
    p, pq = unet.unpack(theta, levels, base), unet.unpack(q, levels, base)
    for name, _, _, k in unet.layer_shapes(levels, base):
        assert np.array_equal(pq[name][1], p[name][1])                    # biases kept
        if k == 3:
            assert np.array_equal(pq[name][0], unet.bf16_round(p[name][0]))
        else:
            assert np.array_equal(pq[name][0], p[name][0])                # the head kept
