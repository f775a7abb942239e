"""Timing of the warm-start network through the C ABI: inference and
training steps on device-resident inputs, timed with CUDA events, and the
convolution FLOP rate.  Prints one JSON line.

    python -m paper_2111_08666_gb300.unet_bench --batch 1 --height 1024 --width 2048
"""
from __future__ import annotations

import json

import numpy as np

from . import mclbm, warmstart


def conv_flops(levels: int, base: int, b: int, h: int, w: int) -> float:
    """2 x 9 x P_l x C_in x C_out summed over the 3x3 convolutions of one
    forward pass (the padded 32 input channels of the first layer)."""
    fl = 0.0
    for name, co, ci, k in warmstart.layer_shapes(levels, base):
        if k != 3:
            continue
        lvl = int(name[3])
        p = b * (h >> lvl) * (w >> lvl)
        fl += 2.0 * 9.0 * p * co * (32 if ci == warmstart.IN_CHANNELS else ci)
    return fl


def main(argv=None) -> None:
    import argparse

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--height", type=int, default=1024)
    ap.add_argument("--width", type=int, default=2048)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--per-tap", action="store_true",
                    help="weight gradients on the per-tap kernel instead of the shared-tap one")
    a = ap.parse_args(argv)
    b, h, w = a.batch, a.height, a.width
    net = mclbm.UNet(a.levels, a.base, max_batch=b, max_h=h, max_w=w)
    if a.per_tap:
        mclbm.mclbm_unet_set_shared_taps(net.h, 0)
    net.set_params(warmstart.init_params(a.levels, a.base, 0))
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.normal(0, 1, (b, h, w, 4)).astype(np.float32)).cuda()
    t = torch.from_numpy(np.tanh(rng.normal(0, 1, (b, h, w))).astype(np.float32)).cuda()
    m = torch.ones((b, h, w), dtype=torch.float32, device="cuda")
    phi = torch.empty((b, h, w), dtype=torch.float32, device="cuda")
    fl = conv_flops(a.levels, a.base, b, h, w)

    def timed(fn):
        for _ in range(a.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / a.reps  # ms (the calls synchronise the network's stream)

    out = dict(levels=a.levels, base=a.base, batch=b, height=h, width=w, forward_gflop=fl / 1e9,
               wgrad="per-tap" if a.per_tap else "shared-tap")
    ms = timed(lambda: mclbm.mclbm_unet_infer(net.h, b, h, w, x, phi))
    out.update(infer_ms=ms, infer_tflops=fl / (ms * 1e-3) / 1e12)
    if not a.no_train:
        ms = timed(lambda: mclbm.mclbm_unet_train_step(net.h, b, h, w, x, t, m, 1e-4))
        out.update(train_ms=ms, train_tflops=3 * fl / (ms * 1e-3) / 1e12)
    print(json.dumps(out))
    net.close()


if __name__ == "__main__":
    main()
