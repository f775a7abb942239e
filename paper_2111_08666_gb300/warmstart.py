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


# --- training pairs from the batched LBM -----------------------------------------

DP_SCALE = 100.0  # input channel 3 = pressure step (inlet density increment) x DP_SCALE


def training_case(seed: int, size: int = 256) -> dict:
    """Medium of the training set: lognormal disks (mean radius 10, sigma_log
    0.4), porosity 0.6, contact angle drawn from U[30, 150] deg with the
    seed, viscosity ratio 10; primary drainage set-up at equal pressures."""
    from . import media
    theta = float(np.random.default_rng(seed).uniform(30.0, 150.0))
    m = media.make_disk_medium(size, size, seed, radius="lognormal", r_mean=10.0, sigma_log=0.4,
                               porosity=0.6)
    rho1, rho2 = media.drainage_densities(m.solid)
    return dict(solid=m.solid, xi=media.uniform_xi(m.solid, media.theta_to_xi(theta)), rho1=rho1,
                rho2=rho2, nu1=(1.7 - 0.5) / 3.0, nu2=(0.62 - 0.5) / 3.0, g_coh=3.5,
                rho_in1=1.0, rho_out2=1.0, theta=theta)


def relax(step, saturation, window: int = 1000, tol: float = 1e-6, max_steps: int = 40000):
    """Step until S_w (by mass) changes by less than tol over one window
    (the convergence reading of Sec. 4.2.1).  Returns (steps, S_w, converged)."""
    prev = saturation()
    n = 0
    while n < max_steps:
        step(window)
        n += window
        cur = saturation()
        if not np.isfinite(cur):
            return n, cur, False
        if abs(cur - prev) < tol:
            return n, cur, True
        prev = cur
    return n, prev, False


def drainage_pairs(seeds, size: int = 256, levels: int = 6, d_rho: float = 0.004,
                   window: int = 1000, tol: float = 1e-6, max_steps: int = 30000, batch: int = 24):
    """Quasi-static primary drainage of the training media with the batched
    kernel: relax at equal pressures, then raise the inlet density of
    component 1 by d_rho per level and relax again.  Returns the network
    inputs [N][size][size][4], targets (phase field after the level) and
    fluid masks, and the relaxation steps of every (case, level)."""
    xs, ts, ms, steps = [], [], [], []
    seeds = list(seeds)
    for c0 in range(0, len(seeds), batch):
        cases = [training_case(s, size) for s in seeds[c0:c0 + batch]]
        b = mclbm.mclbm_batch_create(cases, mclbm.MCLBM_FP32)
        try:
            views = [mclbm.LatticeView(b, k, size, size, mclbm.MCLBM_FP32) for k in range(len(cases))]
            fluid = [(c["solid"] == 0).astype(np.float32) for c in cases]

            def run_level():
                prev = [v.diagnostics()["sw_mass"] for v in views]
                done = [0] * len(views)
                n = 0
                while n < max_steps and not all(done):
                    mclbm.mclbm_batch_step(b, window)
                    n += window
                    cur = [v.diagnostics()["sw_mass"] for v in views]
                    for k in range(len(views)):
                        if not done[k] and abs(cur[k] - prev[k]) < tol:
                            done[k] = n
                    prev = cur
                return [d if d else n for d in done]

            run_level()
            phase = [v.phase() for v in views]
            for lev in range(1, levels + 1):
                for v in views:
                    v.set_pressure_bc(1.0 + lev * d_rho, 1.0)
                st = run_level()
                new = [v.phase() for v in views]
                for k, c in enumerate(cases):
                    xs.append(network_input(c["solid"], c["xi"], phase[k], d_rho * DP_SCALE))
                    ts.append(new[k])
                    ms.append(fluid[k])
                    steps.append(st[k])
                phase = new
        finally:
            mclbm.mclbm_batch_destroy(b)
    return (np.stack(xs).astype(np.float32), np.stack(ts).astype(np.float32),
            np.stack(ms).astype(np.float32), np.array(steps))


def train(net, x, t, m, epochs: int = 10, batch: int = 16, lr: float = 1e-3, seed: int = 0):
    """Adam on the masked MSE, shuffled mini-batches; returns the mean loss
    of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    n = x.shape[0]
    for _ in range(epochs):
        order = rng.permutation(n)
        losses = []
        for i in range(0, n - batch + 1, batch):
            idx = order[i:i + batch]
            losses.append(net.train_step(x[idx], t[idx], m[idx], lr))
        hist.append(float(np.mean(losses)))
    return hist


def drainage_curves(net, case: dict, levels: int = 20, d_rho: float = 0.005, window: int = 1000,
                    tol: float = 1e-6, max_steps: int = 200000, flip: float = 0.0, gate: int = 0,
                    stream=None, warm: bool = True, mrt: bool = False):
    """Quasi-static primary drainage of one lattice (Sec. 4.2.1), run as two
    independent P_c-S_w curves from the same relaxed start:

    cold  each level continues from the curve's previous equilibrium under
          the raised inlet density (the protocol of Sec. 4.2);
    warm  each level starts from the warm curve's own previous equilibrium
          with the network's prediction blended in (``mclbm_blend_phase``:
          the nodes predicted to change phase are reset to the predicted
          phase, every other node keeps its populations), then relaxes.

    The blend is applied only where the network predicts a real invasion:
    at least ``gate`` fluid nodes whose predicted phase lies on the other
    side of zero (by more than ``flip``); a smaller predicted change leaves
    the level to the cold continuation (resetting a few nodes to rest costs
    more relaxation, by the pressure waves it sends, than it saves).  The
    warm wall time of a level counts everything the warm start adds: the
    phase read-out, the network input, the inference and the blend.

    A level ends when |S_w(t) - S_w(t - window)| < tol (S_w by mass) or
    after max_steps; the library's divergence check runs every window, and
    a curve that diverges stops there (its record says so).  ``warm=False``
    runs the cold curve only; ``mrt`` steps both curves with the MRT
    collision (energy rates tied to 1/tau_s, heat-flux rate 1.9) instead of
    the SRT of Eq. 1.  Returns one record per level."""
    import time

    def make():
        lat = mclbm.Lattice(case["solid"], case["xi"], prec="fp32", nu1=case["nu1"],
                            nu2=case["nu2"], rho_in1=case["rho_in1"], rho_out2=case["rho_out2"],
                            stream=stream)
        mclbm.mclbm_set_flag(lat.h, mclbm.MCLBM_FLAG_DIAG_EVERY, window)
        if mrt:
            lat.set_mrt(True, 0.0, 0.0, 1.9)
        lat.init(case["rho1"], case["rho2"])
        return lat

    def relax_checked(lat):
        try:
            n, s_end, ok = relax(lat.step, lambda: sw(lat), window, tol, max_steps)
            lat.sync()  # reports the library's divergence check
            return n, s_end, ok, not np.isfinite(s_end)
        except mclbm.MclbmError as e:
            if e.code != mclbm.MCLBM_ERR_DIVERGED:
                raise
            return None, float("nan"), False, True

    def sw(l):
        return l.diagnostics()["sw_mass"]

    branches = {"cold": make()}
    if warm:
        branches["warm"] = make()
    # the common start: both relax at the initial boundary densities (the
    # kernels are deterministic, so the two states are identical)
    for name, lat in list(branches.items()):
        if relax_checked(lat)[3]:
            raise RuntimeError("the lattice diverged at the initial boundary densities")
    fluid = case["solid"] == 0
    out = []
    for lev in range(1, levels + 1):
        rho_in = case["rho_in1"] + lev * d_rho
        rec = dict(level=lev, rho_in1=rho_in)
        for name, lat in list(branches.items()):
            sw0 = sw(lat)
            t0 = time.perf_counter()
            lat.set_pressure_bc(rho_in, case["rho_out2"])
            if name == "warm":
                phase = lat.phase()
                x = network_input(case["solid"], case["xi"], phase, d_rho * DP_SCALE)[None]
                phi = net.infer(x)[0]
                p = np.clip(phi, -1.0, 1.0)
                predicted = int((fluid & ((p > 0) != (phase > 0)) & (np.abs(p) > flip)).sum())
                rec["nodes_predicted"] = predicted
                rec["nodes_changed"] = mclbm.mclbm_blend_phase(lat.h, phi, flip) if predicted >= gate else 0
                rec["sec_predict"] = time.perf_counter() - t0
            n, s_end, ok, diverged = relax_checked(lat)
            rec.update({f"steps_{name}": n, f"sw_{name}": s_end, f"converged_{name}": ok,
                        f"diverged_{name}": diverged, f"sec_{name}": time.perf_counter() - t0,
                        f"sw_before_{name}": sw0})
            if diverged:
                lat.close()
                del branches[name]
            else:
                rec[f"pc_{name}"] = lat.diagnostics()["pc"]
        out.append(rec)
        if not branches:
            break
    for lat in branches.values():
        lat.close()
    return out


def main(argv=None) -> None:
    """Generate training pairs, train, and compare warm and cold relaxation
    on a large lattice; prints one JSON line."""
    import argparse
    import json
    import time

    from . import media
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-media", type=int, default=300)
    ap.add_argument("--train-levels", type=int, default=6)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--eval-nx", type=int, default=2048)
    ap.add_argument("--eval-ny", type=int, default=1024)
    ap.add_argument("--eval-levels", type=int, default=20)
    ap.add_argument("--max-steps", type=int, default=200000)
    ap.add_argument("--train-max-steps", type=int, default=30000)
    ap.add_argument("--d-rho", type=float, default=0.005)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--flip", type=float, default=0.0)
    ap.add_argument("--gates", type=str, default="1000",
                    help="comma list of gates: predicted flipped nodes below which a level is left to "
                         "the cold continuation (one evaluation per gate, the same trained network)")
    ap.add_argument("--mrt", action="store_true",
                    help="step both evaluation curves with the MRT collision (training pairs stay SRT)")
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    x, t, m, st = drainage_pairs(range(1000, 1000 + a.train_media), levels=a.train_levels,
                                 d_rho=a.d_rho, tol=a.tol, max_steps=a.train_max_steps)
    t_data = time.perf_counter() - t0
    net = mclbm.UNet(4, 32, max_batch=16, max_h=256, max_w=256)
    net.set_params(init_params(4, 32, 0))
    t0 = time.perf_counter()
    hist = train(net, x, t, m, epochs=a.epochs)
    t_train = time.perf_counter() - t0
    big = mclbm.UNet(4, 32, max_batch=1, max_h=a.eval_ny, max_w=a.eval_nx)
    big.set_params(net.params())
    net.close()
    case = media.config_paper_scale(a.eval_nx, a.eval_ny, 99)
    for gate in [int(g) for g in a.gates.split(",")]:
        rec = drainage_curves(big, case, levels=a.eval_levels, d_rho=a.d_rho, tol=a.tol,
                              max_steps=a.max_steps, flip=a.flip, gate=gate, mrt=a.mrt)
        both = [r for r in rec if r.get("steps_cold") and r.get("steps_warm")]
        summary = dict(gate=gate, mrt=a.mrt, train_pairs=int(x.shape[0]), data_sec=t_data, train_sec=t_train,
                       loss=hist,
                       pair_steps_mean=float(st.mean()),
                       levels_compared=len(both),
                       steps_cold=int(sum(r["steps_cold"] for r in both)),
                       steps_warm=int(sum(r["steps_warm"] for r in both)),
                       sec_cold=float(sum(r["sec_cold"] for r in both)),
                       sec_warm=float(sum(r["sec_warm"] for r in both)),
                       levels_unconverged_cold=int(sum(not r["converged_cold"] for r in both)),
                       levels_unconverged_warm=int(sum(not r["converged_warm"] for r in both)),
                       diverged=[(r["level"], k) for r in rec for k in ("cold", "warm")
                                 if r.get(f"diverged_{k}")],
                       max_abs_dsw=float(max(abs(r["sw_cold"] - r["sw_warm"]) for r in both)) if both else None,
                       levels=rec)
        print(json.dumps(summary), flush=True)
    big.close()


if __name__ == "__main__":
    main()
