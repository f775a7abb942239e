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
