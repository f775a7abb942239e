"""Plain FP64 NumPy reference of the warm-start U-Net: forward, backward and
loss, written as the textbook operations (3x3 convolutions by shifted
matrix products, 2x2 average pooling, nearest upsampling, channel concat,
ReLU, tanh, masked mean squared error).

TEST INFRASTRUCTURE ONLY: the GPU network is checked against this module;
the product never imports it.

Network (levels L, base channels C0, channels C_l = C0 * 2^l):
  encoder l = 0..L-1:  conv3x3(C_in -> C_l) + ReLU, conv3x3(C_l -> C_l) + ReLU
                       = e_l; 2x2 average pooling feeds level l+1
                       (C_in = 8 at level 0: 4 input channels padded with 4 zeros)
  decoder l = L-2..0:  concat(e_l, nearest-upsample(d_{l+1})) (skip first),
                       conv3x3(C_l + C_{l+1} -> C_l) + ReLU, conv3x3(C_l -> C_l)
                       + ReLU = d_l   (d_{L-1} = e_{L-1})
  head:                1x1 conv C0 -> 1, tanh
Loss: mean over the masked (fluid) pixels of (phi_hat - phi_target)^2.

Parameters, flat and in this order, each conv as weights [Co][3][3][Ci]
(1x1 for the head: [1][C0]) followed by its bias [Co]: enc0a, enc0b, ...,
enc(L-1)a, enc(L-1)b, dec(L-2)a, dec(L-2)b, ..., dec0a, dec0b, head.
Tensors are NHWC.

Storage model (optional).  The network is defined with BF16 storage: its
input, its 3x3 weights and every activation it keeps (each conv output
after ReLU, each pooled map) are bfloat16 values, and so is, in the
backward pass, every gradient at a conv's pre-activation (after the ReLU
mask), from which that conv's weight and input gradients are formed;
biases, the head and all sums are wider.  ``forward(..., store=bf16_round)`` together with
``store_weights`` evaluates exactly that network in FP64: the values are
rounded where the storage format rounds them, so that the ReLU masks (a
discrete outcome that a 2^-9 perturbation can flip) are decided on the same
values as in a BF16 implementation.  With ``store=None`` every function is
the plain FP64 network.
"""
from __future__ import annotations

import numpy as np

IN_CHANNELS = 8


def layer_shapes(levels: int, base: int):
    """(name, C_out, C_in, kernel) of every conv in parameter order."""
    ch = [base * (1 << l) for l in range(levels)]
    out = []
    for l in range(levels):
        cin = IN_CHANNELS if l == 0 else ch[l - 1]
        out.append((f"enc{l}a", ch[l], cin, 3))
        out.append((f"enc{l}b", ch[l], ch[l], 3))
    for l in range(levels - 2, -1, -1):
        out.append((f"dec{l}a", ch[l], ch[l] + ch[l + 1], 3))
        out.append((f"dec{l}b", ch[l], ch[l], 3))
    out.append(("head", 1, base, 1))
    return out


def param_count(levels: int, base: int) -> int:
    return sum(co * k * k * ci + co for _, co, ci, k in layer_shapes(levels, base))


def unpack(theta: np.ndarray, levels: int, base: int):
    params, o = {}, 0
    for name, co, ci, k in layer_shapes(levels, base):
        n = co * k * k * ci
        params[name] = (theta[o:o + n].reshape(co, k, k, ci), theta[o + n:o + n + co])
        o += n + co
    assert o == theta.size
    return params


def pack(grads: dict, levels: int, base: int) -> np.ndarray:
    parts = []
    for name, co, ci, k in layer_shapes(levels, base):
        gw, gb = grads[name]
        parts += [gw.reshape(-1), gb.reshape(-1)]
    return np.concatenate(parts)


def bf16_round(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even),
    returned as float64.  Values are first rounded to float32, the type a
    BF16 implementation converts from."""
    u = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32)).view(np.uint32)
    u = u.astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def store_weights(theta, levels: int, base: int, rnd=bf16_round) -> np.ndarray:
    """The parameter vector with every 3x3 weight rounded by ``rnd``; the
    biases and the head (1x1) are kept."""
    out = np.array(theta, np.float64, copy=True)
    o = 0
    for name, co, ci, k in layer_shapes(levels, base):
        n = co * k * k * ci
        if k == 3:
            out[o:o + n] = rnd(out[o:o + n])
        o += n + co
    return out


def conv3(x, w, b):
    """3x3 convolution, zero padding 1: y[p] = sum_{dy,dx} x[p+d] W[:,dy,dx,:]^T + b."""
    bsz, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((bsz, h, wd, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + h, kx:kx + wd, :] @ w[:, ky, kx, :].T
    return y + b


def conv3_backward(x, w, dy):
    """Gradients of conv3 with respect to x, w and b."""
    bsz, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            xs = xp[:, ky:ky + h, kx:kx + wd, :]
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwi->oi", dy, xs)
            dxp[:, ky:ky + h, kx:kx + wd, :] += dy @ w[:, ky, kx, :]
    return dxp[:, 1:h + 1, 1:wd + 1, :], dw, dy.sum(axis=(0, 1, 2))


def pool2(x):
    b, h, w, c = x.shape
    return x.reshape(b, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(dy):
    b, h, w, c = dy.shape
    return dy.reshape(b, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def forward(theta, x, levels: int, base: int, store=None):
    """Returns phi_hat [B][H][W] and the cache for backward.  ``store`` (see
    the storage model above) rounds the input and every kept activation."""
    keep = store if store is not None else (lambda a: a)
    p = unpack(theta, levels, base)
    cache = {}
    e, h = [], keep(x)
    for l in range(levels):
        if l > 0:
            h = keep(pool2(e[-1]))
        a_in = h
        za = conv3(a_in, *p[f"enc{l}a"])
        ha = keep(np.maximum(za, 0.0))
        zb = conv3(ha, *p[f"enc{l}b"])
        hb = keep(np.maximum(zb, 0.0))
        cache[f"enc{l}"] = (a_in, za, ha, zb)
        e.append(hb)
    d = e[-1]
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([e[l], up2(d)], axis=3)
        za = conv3(cat, *p[f"dec{l}a"])
        ha = keep(np.maximum(za, 0.0))
        zb = conv3(ha, *p[f"dec{l}b"])
        d = keep(np.maximum(zb, 0.0))
        cache[f"dec{l}"] = (cat, za, ha, zb)
    hw, hb = p["head"]
    z = d @ hw[:, 0, 0, :].T + hb
    phi = np.tanh(z[..., 0])
    cache["head"] = (d, phi)
    cache["e"] = e
    return phi, cache


def loss_and_grad_phi(phi, target, mask):
    n = max(float(mask.sum()), 1.0)
    r = (phi - target) * mask
    return float((r * r).sum() / n), 2.0 * r / n


def backward(theta, cache, dphi, levels: int, base: int, store=None) -> np.ndarray:
    keep = store if store is not None else (lambda a: a)
    p = unpack(theta, levels, base)
    grads = {}
    d, phi = cache["head"]
    hw, _ = p["head"]
    dz = (dphi * (1.0 - phi * phi))[..., None]
    grads["head"] = (np.einsum("bhwo,bhwi->oi", dz, d)[:, None, None, :], dz.sum(axis=(0, 1, 2)))
    dd = dz @ hw[:, 0, 0, :]
    e = cache["e"]
    de = [np.zeros_like(t) for t in e]
    for l in range(0, levels - 1):
        cat, za, ha, zb = cache[f"dec{l}"]
        dzb = keep(dd * (zb > 0))
        dha, gw, gb = conv3_backward(ha, p[f"dec{l}b"][0], dzb)
        grads[f"dec{l}b"] = (gw, gb)
        dza = keep(dha * (za > 0))
        dcat, gw, gb = conv3_backward(cat, p[f"dec{l}a"][0], dza)
        grads[f"dec{l}a"] = (gw, gb)
        c_skip = e[l].shape[3]
        de[l] += dcat[..., :c_skip]
        dd = up2_backward(dcat[..., c_skip:])
    de[levels - 1] += dd
    for l in range(levels - 1, -1, -1):
        a_in, za, ha, zb = cache[f"enc{l}"]
        dzb = keep(de[l] * (zb > 0))
        dha, gw, gb = conv3_backward(ha, p[f"enc{l}b"][0], dzb)
        grads[f"enc{l}b"] = (gw, gb)
        dza = keep(dha * (za > 0))
        dx, gw, gb = conv3_backward(a_in, p[f"enc{l}a"][0], dza)
        grads[f"enc{l}a"] = (gw, gb)
        if l > 0:
            de[l - 1] += pool2_backward(dx)
    return pack(grads, levels, base)


def loss_and_gradient(theta, x, target, mask, levels: int, base: int, store=None):
    phi, cache = forward(theta, x, levels, base, store)
    loss, dphi = loss_and_grad_phi(phi, target, mask)
    return loss, backward(theta, cache, dphi, levels, base, store), phi
