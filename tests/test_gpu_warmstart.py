"""What the trained warm-start network gains (the learned warm start of the
quasi-static drainage protocol, Sec. 4.2.1): a network briefly trained on
LBM equilibria of small media cuts the relaxation steps of a drainage curve
on an unseen medium against the cold-started curve, reaching the same
saturations (|dS_w| <= 0.005 per level); the same network untrained does
not (more steps, other saturations, or a curve that diverges).  Everything runs through the C ABI:
training pairs from the batched LBM, training and inference on the
tensor-core U-Net, the blend in the library."""
import numpy as np
import pytest

from paper_2111_08666_gb300 import mclbm, warmstart

pytestmark = pytest.mark.gpu

LEVELS, D_RHO = 3, 0.01
RELAX = dict(window=1000, tol=1e-6)


def _curves(params, case):
    net = mclbm.UNet(4, 32, max_batch=1, max_h=256, max_w=256)
    net.set_params(params)
    rec = warmstart.drainage_curves(net, case, levels=LEVELS, d_rho=D_RHO, max_steps=100000,
                                    **RELAX)
    net.close()
    assert len(rec) == LEVELS and not any(r.get("diverged_cold") for r in rec)
    cold = sum(r["steps_cold"] for r in rec)
    if any(r.get("diverged_warm") for r in rec):   # a curve that diverges gains nothing
        return cold, float("inf"), float("inf"), rec
    warm = sum(r["steps_warm"] for r in rec)
    dsw = max(abs(r["sw_cold"] - r["sw_warm"]) for r in rec)
    return cold, warm, dsw, rec


def test_trained_network_gains_over_cold_and_untrained_starts():
    # 48 media of 128 x 128 (seeds 1000-1047, theta ~ U[30, 150] deg), three
    # drainage levels each, relaxed by the batched LBM
    x, t, m, _ = warmstart.drainage_pairs(range(1000, 1048), size=128, levels=LEVELS, d_rho=D_RHO,
                                          max_steps=50000, batch=24, **RELAX)
    net = mclbm.UNet(4, 32, max_batch=16, max_h=128, max_w=128)
    init = warmstart.init_params(4, 32, 0)
    net.set_params(init)
    hist = warmstart.train(net, x, t, m, epochs=30, batch=16, lr=1e-3)
    trained = net.params()
    net.close()
    assert hist[-1] < 0.2 * hist[0]
    case = warmstart.training_case(5000, 256)       # a medium outside the training set
    cold, warm, dsw, rec = _curves(trained, case)
    print("trained:", cold, warm, dsw, [(r["steps_cold"], r["steps_warm"], r["nodes_changed"]) for r in rec])
    assert warm < cold
    assert dsw <= 0.005
    cold0, warm0, dsw0, _ = _curves(init, case)
    print("untrained:", cold0, warm0, dsw0)
    assert cold0 == cold                             # the cold curve does not use the network
    assert warm0 > warm or dsw0 > 0.005
