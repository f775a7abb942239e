"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: FP64 populations within 1e-10 of max|f| after 200+ steps; FP32
densities within 1e-4 and saturation within 1e-3 (absolute).  Inputs are the
seeded synthetic media of ``paper_2111_08666_gb300.media``; the oracle and
the GPU start from the same arrays.
"""
import numpy as np
import pytest

import oracle
from paper_2111_08666_gb300 import media
from paper_2111_08666_gb300 import mclbm

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def nu_of_tau(t):
    return (t - 0.5) / 3.0


KERNELS = {"tile": 1, "strip": 2}


@pytest.fixture(params=list(KERNELS))
def kernel(request):
    return KERNELS[request.param]


def pair(solid, xi, rho1, rho2, prec="fp64", kernel=0, **kw):
    """The same case on the oracle and on the GPU."""
    o = oracle.Oracle(solid, xi, **kw)
    o.init(rho1, rho2)
    g = mclbm.Lattice(solid, xi, prec=prec, kernel=kernel, **kw)
    g.init(rho1, rho2)
    return o, g


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def assert_fp64_parity(o, g, steps):
    o.step(steps)
    g.step(steps)
    f = g.populations()
    err = rel_err(f, o.f)
    assert err < FP64_TOL, err
    return f


def test_init_and_roundtrip_exact():
    c = media.config_small_fp64()
    o, g = pair(c["solid"], c["xi"], c["rho1"], c["rho2"], nu1=c["nu1"], nu2=c["nu2"],
                rho_in1=1.01, rho_out2=1.0)
    f = g.populations()
    assert np.array_equal(f, o.f)
    rng = np.random.default_rng(0)
    h = rng.random(f.shape) * (c["solid"] == 0)
    g.set_populations(h)
    assert np.array_equal(g.populations(), h)


def test_fp64_disk_medium_drainage_200_steps(kernel):
    """128x64 disk medium, radii U[4,8], porosity ~0.65, Set-3 boundaries
    with rho_in = 1.01, rho_out = 1, neutral wetting, M = 1."""
    c = media.config_small_fp64()
    o, g = pair(c["solid"], c["xi"], c["rho1"], c["rho2"], kernel=kernel, nu1=c["nu1"], nu2=c["nu2"],
                rho_in1=c["rho_in1"], rho_out2=c["rho_out2"])
    assert_fp64_parity(o, g, 200)
    assert_fp64_parity(o, g, 300)  # 500 in total


def test_fp64_ragged_mixed_wettability_viscosity_ratio_25(kernel):
    """Sizes off every tile multiple, several per-site xi values, M = 25."""
    nx, ny = 45, 21
    m = media.make_disk_medium(nx, ny, 7, radius="uniform", r_lo=2.0, r_hi=4.0,
                               porosity=0.75, reservoir=5)
    rng = np.random.default_rng(1)
    xi = np.where(m.solid != 0, rng.choice([-0.55, -0.4, 0.0, 0.2, 0.5], size=m.solid.shape),
                  0.0).astype(np.float32)
    rho1, rho2 = media.drainage_densities(m.solid, oil_columns=4)
    o, g = pair(m.solid, xi, rho1, rho2, kernel=kernel, nu1=nu_of_tau(3.5), nu2=nu_of_tau(0.62),
                rho_in1=1.02, rho_out2=1.0)
    assert_fp64_parity(o, g, 300)


def test_fp64_periodic_droplet_with_grain_and_body_force(kernel):
    nx, ny = 40, 30
    solid = np.zeros((ny, nx), np.uint8)
    yy, xx = np.mgrid[0:ny, 0:nx]
    solid[(xx - 28) ** 2 + (yy - 15) ** 2 <= 20] = 1
    xi = media.uniform_xi(solid, 0.3)
    rho1, rho2 = media.droplet_densities(nx, ny, 12, 14, 6, solid=solid)
    o, g = pair(solid, xi, rho1, rho2, kernel=kernel, nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62),
                periodic_y=True, gx=2e-5, gy=-1e-5)
    assert_fp64_parity(o, g, 250)


def test_fp64_open_x_periodic_y(kernel):
    nx, ny = 50, 24
    solid = np.zeros((ny, nx), np.uint8)
    solid[8:14, 20:27] = 1
    xi = media.uniform_xi(solid, -0.3)
    rho1, rho2 = media.drainage_densities(solid)
    o, g = pair(solid, xi, rho1, rho2, kernel=kernel, nu1=nu_of_tau(1.0), nu2=nu_of_tau(0.62),
                rho_in1=1.015, rho_out2=1.0, periodic_y=True)
    assert_fp64_parity(o, g, 200)


def test_fp64_unshifted_velocity_reading(kernel):
    nx, ny = 37, 19
    m = media.make_disk_medium(nx, ny, 3, radius="uniform", r_lo=2.0, r_hi=3.0,
                               porosity=0.8, reservoir=4)
    rho1, rho2 = media.drainage_densities(m.solid, oil_columns=3)
    o, g = pair(m.solid, media.uniform_xi(m.solid, -0.2), rho1, rho2, kernel=kernel, nu1=0.1,
                nu2=0.05,
                rho_in1=1.01, rho_out2=1.0, vel_shift=False)
    assert_fp64_parity(o, g, 200)


def test_fp64_lattice_smaller_than_a_tile(kernel):
    nx, ny = 7, 5
    solid = np.zeros((ny, nx), np.uint8)
    solid[2, 3] = 1
    rng = np.random.default_rng(5)
    rho1 = (0.1 + rng.random((ny, nx))) * (solid == 0)
    rho2 = (0.1 + rng.random((ny, nx))) * (solid == 0)
    o, g = pair(solid, media.uniform_xi(solid, 0.1), rho1, rho2, kernel=kernel, nu1=0.12,
                nu2=0.2,
                periodic_y=True)
    assert_fp64_parity(o, g, 200)


def test_readouts_and_diagnostics_match_oracle(kernel):
    c = media.config_small_fp64()
    o, g = pair(c["solid"], media.uniform_xi(c["solid"], -0.4), c["rho1"], c["rho2"],
                kernel=kernel, nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), rho_in1=1.01, rho_out2=1.0)
    o.step(150)
    g.step(150)
    assert rel_err(g.density(), o.density()) < FP64_TOL
    ux, uy = g.velocity()
    umax = max(np.abs(o.ux).max(), np.abs(o.uy).max())
    assert np.max(np.abs(ux - o.ux)) < 1e-9 * umax
    assert np.max(np.abs(uy - o.uy)) < 1e-9 * umax
    assert rel_err(g.pressure(), o.pressure_field()) < FP64_TOL
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass1", "mass2", "sw_mass", "p_in", "p_out"):
        assert dg[k] == pytest.approx(do[k], rel=1e-12), k
    assert dg["sw_count"] == do["sw_count"]
    assert dg["n_fluid"] == do["n_fluid"]
    assert dg["pc"] == pytest.approx(do["pc"], abs=1e-13)
    rho = o.density()
    phase = np.where(c["solid"] == 0, (rho[0] - rho[1]) / np.maximum(rho[0] + rho[1], 1e-300), 0)
    assert np.max(np.abs(g.phase() - phase)) < 1e-6


def test_fp32_matches_oracle_after_1e4_steps_stable_case():
    """The FP32 bar (densities 1e-4, saturation 1e-3 absolute after 10^4
    steps) on the 128x64 disk medium with balanced boundary densities: the
    interfaces relax to rest instead of invading, so rounding differences
    are not amplified by pore-scale instabilities."""
    c = media.config_small_fp64()
    o, g = pair(c["solid"], c["xi"], c["rho1"], c["rho2"], prec="fp32", nu1=c["nu1"],
                nu2=c["nu2"], rho_in1=1.0, rho_out2=1.0)
    o.step(10000)
    g.step(10000)
    assert rel_err(g.density(), o.density()) < 1e-4
    dg, do = g.diagnostics(), o.diagnostics()
    assert abs(dg["sw_count"] - do["sw_count"]) <= 1e-3
    assert abs(dg["sw_mass"] - do["sw_mass"]) <= 1e-3


def test_fp32_driven_drainage_divergence_growth():
    """Driven drainage (rho_in = 1.01) is unstable at the pore scale, so the
    FP32/FP64 difference grows with time; saturation stays within 1e-3 and
    the density difference within 1e-3 after 2000 steps."""
    c = media.config_small_fp64()
    o, g = pair(c["solid"], c["xi"], c["rho1"], c["rho2"], prec="fp32", nu1=c["nu1"],
                nu2=c["nu2"], rho_in1=c["rho_in1"], rho_out2=c["rho_out2"])
    errs = []
    for _ in range(4):
        o.step(500)
        g.step(500)
        errs.append(rel_err(g.density(), o.density()))
    print("fp32 driven drainage density error at 500..2000 steps:", errs)
    assert errs[-1] < 1e-3
    dg, do = g.diagnostics(), o.diagnostics()
    assert abs(dg["sw_count"] - do["sw_count"]) <= 1e-3
    assert abs(dg["sw_mass"] - do["sw_mass"]) <= 1e-3


def test_mass_conserved_on_gpu_closed_box():
    nx, ny = 64, 40
    solid = np.zeros((ny, nx), np.uint8)
    solid[:2] = 1
    solid[-2:] = 1
    solid[15:25, 40:50] = 1
    rho1, rho2 = media.droplet_densities(nx, ny, 20, 20, 8, solid=solid)
    g = mclbm.Lattice(solid, media.uniform_xi(solid, -0.4), prec="fp64",
                      nu1=nu_of_tau(3.5), nu2=nu_of_tau(0.62))
    g.init(rho1, rho2)
    d0 = g.diagnostics()
    g.step(3000)
    d1 = g.diagnostics()
    assert abs(d1["mass1"] / d0["mass1"] - 1) < 1e-12
    assert abs(d1["mass2"] / d0["mass2"] - 1) < 1e-12


def test_all_solid_lattice_has_no_fluid():
    solid = np.ones((6, 9), np.uint8)
    g = mclbm.Lattice(solid, prec="fp32")
    g.init(np.zeros((6, 9)), np.zeros((6, 9)))
    g.step(3)
    d = g.diagnostics()
    assert d["n_fluid"] == 0 and d["mass1"] == 0
    assert np.isnan(d["sw_count"]) and np.isnan(d["p_in"])


def test_errors_are_reported():
    solid = np.zeros((8, 8), np.uint8)    # fluid on the edge rows, not periodic
    g = mclbm.Lattice(solid, prec="fp32")
    with pytest.raises(mclbm.MclbmError) as e:
        g.step(1)                           # not initialised
    assert e.value.code == mclbm.MCLBM_ERR_STATE
    g.init(np.ones((8, 8)), np.ones((8, 8)))
    with pytest.raises(mclbm.MclbmError) as e:
        g.step(1)                           # rows 0 and ny-1 must be walls
    assert e.value.code == mclbm.MCLBM_ERR_ARG
    xi = np.arange(64, dtype=np.float32).reshape(8, 8) / 1000
    many = np.ones((8, 8), np.uint8)
    with pytest.raises(mclbm.MclbmError):
        mclbm.Lattice(np.ones((20, 20), np.uint8), np.arange(400, dtype=np.float32).reshape(20, 20))
    mclbm.Lattice(many, xi).close()     # 64 distinct values are fine


def test_divergence_flag():
    nx, ny = 16, 16
    solid = np.zeros((ny, nx), np.uint8)
    g = mclbm.Lattice(solid, prec="fp32", periodic_y=True, nu1=0.1, nu2=0.1)
    rho = np.ones((ny, nx))
    rho[5, 5] = -3.0                       # a negative density is caught
    g.init(rho, np.ones((ny, nx)))
    mclbm.mclbm_set_flag(g.h, mclbm.MCLBM_FLAG_DIAG_EVERY, 1)
    g.step(1)
    with pytest.raises(mclbm.MclbmError) as e:
        g.sync()
    assert e.value.code == mclbm.MCLBM_ERR_DIVERGED
    g.sync()                               # the flag is cleared once reported


def test_boundary_mode_switch_keeps_parity(kernel):
    """Switching between periodic x and the Set-3 boundaries mid-run (the
    ghost columns of the strip kernel are rebuilt) matches the oracle."""
    c = media.config_small_fp64()
    o, g = pair(c["solid"], c["xi"], c["rho1"], c["rho2"], kernel=kernel, nu1=c["nu1"],
                nu2=c["nu2"])
    assert_fp64_parity(o, g, 60)
    o.set_pressure_bc(1.01, 1.0)
    g.set_pressure_bc(1.01, 1.0)
    assert_fp64_parity(o, g, 60)
    o.set_pressure_bc(-1, -1)
    g.set_pressure_bc(-1, -1)
    assert_fp64_parity(o, g, 60)


# Agreement of two step formulations, relative to max|f|: one step from the
# same developed state (a few units in the last place of the storage), and
# 300 steps from the initial state (rounding differences of the FP32
# arithmetic, flipped roundings of a 16-bit storage, carried along).
AGREE = {"fp32": (1e-6, 4e-6), "fp32dev": (1e-6, 4e-6), "fp16dev": (1e-4, 1e-3),
         "bf16dev": (1e-3, 4e-3)}


@pytest.mark.parametrize("other", [2, 3, 4])
@pytest.mark.parametrize("prec", ["fp32", "fp32dev", "fp16dev", "bf16dev"])
def test_step_kernels_agree(prec, other):
    """The formulations of the step (global-pull tile, strip, TMA tile,
    fluid-only) compute the same update of Eqs. 1-29 in every storage
    precision; they differ only in data movement and in how the compiler
    fuses the FP32 multiply-adds, so they agree to rounding."""
    if other == 4 and prec == "fp32dev":
        pytest.skip("the fluid-only kernel serves FP32 and the 16-bit storages")
    m = media.make_disk_medium(200, 70, 11, radius="uniform", r_lo=3.0, r_hi=6.0,
                               porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.4)
    rho1, rho2 = media.drainage_densities(m.solid)
    kw = dict(prec=prec, nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), rho_in1=1.01, rho_out2=1.0)
    one, many = AGREE[prec]
    base = mclbm.Lattice(m.solid, xi, kernel=1, **kw)
    base.init(rho1, rho2)
    base.step(200)
    f0 = base.populations()
    a = mclbm.Lattice(m.solid, xi, kernel=1, **kw)
    b = mclbm.Lattice(m.solid, xi, kernel=other, **kw)
    a.set_populations(f0)
    b.set_populations(f0)
    a.step(1)
    b.step(1)
    scale = np.max(np.abs(f0))
    assert np.max(np.abs(a.populations() - b.populations())) <= one * scale
    a.init(rho1, rho2)
    b.init(rho1, rho2)
    a.step(300)
    b.step(300)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) <= many * np.max(np.abs(fa))


# --- inlet/outlet treatments Set-1 and Set-2 (Sec. 2.3) ------------------------

BC_SETS = {1: dict(bc_set=1, rho_in2=0.03, rho_out1=0.025), 2: dict(bc_set=2)}


@pytest.mark.parametrize("bc_set", [1, 2])
def test_fp64_bc_sets_match_oracle(kernel, bc_set):
    """The 128x64 disk medium of the FP64 parity case under Set-1 (Zou-He for
    both components, the other component's densities fixed) and Set-2
    (Eqs. 26-27 frozen from initialisation)."""
    c = media.config_small_fp64()
    o, g = pair(c["solid"], c["xi"], c["rho1"], c["rho2"], kernel=kernel, nu1=c["nu1"], nu2=c["nu2"],
                rho_in1=c["rho_in1"], rho_out2=c["rho_out2"], **BC_SETS[bc_set])
    assert_fp64_parity(o, g, 200)


@pytest.mark.parametrize("bc_set", [1, 2])
def test_fp32_bc_sets_match_oracle(bc_set):
    """FP32 (automatic kernel) against the oracle on the drainage medium
    with viscosity ratio 10, 1000 steps: densities within 1e-4."""
    m = media.make_disk_medium(160, 64, 7, radius="uniform", r_lo=3.0, r_hi=6.0, porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.4)
    rho1, rho2 = media.drainage_densities(m.solid)
    o, g = pair(m.solid, xi, rho1, rho2, prec="fp32", nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62),
                rho_in1=1.01, rho_out2=1.0, **BC_SETS[bc_set])
    o.step(1000)
    g.step(1000)
    want = np.stack([o.f[0].sum(axis=0), o.f[1].sum(axis=0)])
    got = g.density()
    assert np.max(np.abs(got - want)) < 1e-4


@pytest.mark.parametrize("other", [2, 3, 4])
@pytest.mark.parametrize("bc_set", [1, 2])
def test_bc_sets_step_kernels_agree(bc_set, other):
    """Every step kernel applies Set-1 and Set-2 alike (FP32, to rounding)."""
    m = media.make_disk_medium(150, 60, 13, radius="uniform", r_lo=3.0, r_hi=6.0, porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.4)
    rho1, rho2 = media.drainage_densities(m.solid)
    kw = dict(prec="fp32", nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), rho_in1=1.01, rho_out2=1.0,
              **BC_SETS[bc_set])
    a = mclbm.Lattice(m.solid, xi, kernel=1, **kw)
    b = mclbm.Lattice(m.solid, xi, kernel=other, **kw)
    a.init(rho1, rho2)
    b.init(rho1, rho2)
    a.step(300)
    b.step(300)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) <= AGREE["fp32"][1] * np.max(np.abs(fa))


# --- multiple-relaxation-time collision (not in the paper) ------------------------

MRT = dict(mrt=True, s_e=1.1, s_eps=1.2, s_q=-1.0)


def test_fp64_mrt_matches_oracle(kernel):
    """The MRT variant (closed-form moments on the GPU, the matrix form in
    the oracle) on the FP64 disk-medium drainage case at viscosity ratio 25."""
    c = media.config_small_fp64()
    o, g = pair(c["solid"], media.uniform_xi(c["solid"], -0.3), c["rho1"], c["rho2"], kernel=kernel,
                nu1=nu_of_tau(3.5), nu2=nu_of_tau(0.62), rho_in1=c["rho_in1"], rho_out2=c["rho_out2"],
                **MRT)
    assert_fp64_parity(o, g, 200)


@pytest.mark.parametrize("other", [2, 3, 4])
def test_mrt_step_kernels_agree(other):
    """Every step kernel collides alike under MRT (FP32, to rounding)."""
    m = media.make_disk_medium(150, 60, 17, radius="uniform", r_lo=3.0, r_hi=6.0, porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.4)
    rho1, rho2 = media.drainage_densities(m.solid)
    kw = dict(prec="fp32", nu1=nu_of_tau(3.5), nu2=nu_of_tau(0.62), rho_in1=1.01, rho_out2=1.0, **MRT)
    a = mclbm.Lattice(m.solid, xi, kernel=1, **kw)
    b = mclbm.Lattice(m.solid, xi, kernel=other, **kw)
    a.init(rho1, rho2)
    b.init(rho1, rho2)
    a.step(300)
    b.step(300)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) <= AGREE["fp32"][1] * np.max(np.abs(fa))


def test_mrt_with_tied_rates_is_the_srt_step():
    c = media.config_small_fp64()
    kw = dict(prec="fp64", nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), rho_in1=1.01, rho_out2=1.0)
    a = mclbm.Lattice(c["solid"], c["xi"], **kw)
    b = mclbm.Lattice(c["solid"], c["xi"], mrt=True, **kw)
    a.init(c["rho1"], c["rho2"])
    b.init(c["rho1"], c["rho2"])
    a.step(200)
    b.step(200)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) < 1e-12 * np.max(np.abs(fa))


@pytest.mark.parametrize("periodic_y,open_x", [(True, False), (True, True), (False, False)])
def test_tma_kernel_ghost_frames_fp32(periodic_y, open_x):
    """The TMA tile kernel reads its ring from the ghost columns and rows at
    periodic edges; a lattice off every tile multiple, against the oracle."""
    nx, ny = 75, 41
    solid = np.zeros((ny, nx), np.uint8)
    if not periodic_y:
        solid[0] = solid[-1] = 1
    yy, xx = np.mgrid[0:ny, 0:nx]
    solid[(xx - 50) ** 2 + (yy - 20) ** 2 <= 30] = 1
    xi = media.uniform_xi(solid, -0.3)
    rho1, rho2 = media.droplet_densities(nx, ny, 20, 20, 9, solid=solid)
    kw = dict(nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), periodic_y=periodic_y)
    if open_x:
        rho1, rho2 = media.drainage_densities(solid)
        kw.update(rho_in1=1.01, rho_out2=1.0)
    o, g = pair(solid, xi, rho1, rho2, prec="fp32", kernel=3, **kw)
    o.step(300)
    g.step(300)
    assert rel_err(g.populations(), o.f) < 2e-5


@pytest.mark.parametrize("prec", ["fp32", "fp32dev", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("open_x", [False, True])
def test_tile_shapes_agree(prec, open_x):
    """The two tile shapes of the TMA kernel (32 x 16 or 32 x 12, and 32 x 8)
    cut the lattice differently but compute the same update, on a lattice
    off every tile multiple."""
    nx, ny = 75, 41
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    yy, xx = np.mgrid[0:ny, 0:nx]
    solid[(xx - 50) ** 2 + (yy - 20) ** 2 <= 30] = 1
    xi = media.uniform_xi(solid, -0.3)
    kw = dict(prec=prec, nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), kernel=3)
    if open_x:
        rho1, rho2 = media.drainage_densities(solid)
        kw.update(rho_in1=1.01, rho_out2=1.0)
    else:
        rho1, rho2 = media.droplet_densities(nx, ny, 20, 20, 9, solid=solid)
    a = mclbm.Lattice(solid, xi, tile_shape=0, **kw)
    b = mclbm.Lattice(solid, xi, tile_shape=1, **kw)
    a.init(rho1, rho2)
    b.init(rho1, rho2)
    a.step(200)
    b.step(200)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) <= AGREE[prec][1] * np.max(np.abs(fa))


@pytest.mark.parametrize("prec,bc_set", [("fp32", 3), ("bf16dev", 3), ("fp64", 3), ("fp32", 2)])
def test_checkpoint_restores_bit_for_bit(prec, bc_set, tmp_path):
    """A run saved and loaded into another lattice (created with other
    parameters) continues exactly as the original (with Set-2 this needs the
    frozen inlet values of Eq. 27 restored as well)."""
    m = media.make_disk_medium(96, 48, 4, radius="uniform", r_lo=3.0, r_hi=6.0, porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.3)
    rho1, rho2 = media.drainage_densities(m.solid)
    a = mclbm.Lattice(m.solid, xi, prec=prec, nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62),
                      rho_in1=1.01, rho_out2=1.0, bc_set=bc_set)
    a.init(rho1, rho2)
    a.step(40)
    path = tmp_path / "state.ckpt"
    mclbm.mclbm_save(a.h, path)
    b = mclbm.Lattice(m.solid, xi, prec=prec)  # default parameters, periodic x
    mclbm.mclbm_load(b.h, path)
    assert b.info()["steps"] == a.info()["steps"] == 40
    a.step(40)
    b.step(40)
    assert np.array_equal(a.populations(), b.populations())
    other = mclbm.Lattice(m.solid[:, :64], xi[:, :64], prec=prec)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_load(other.h, path)



@pytest.mark.parametrize("tile_shape", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("periodic_y,open_x", [(True, False), (True, True), (False, False),
                                               (False, True)])
def test_fluid_only_kernel_ragged_lattice(prec, periodic_y, open_x, tile_shape):
    """Kernel 4 stages ring nodes across periodic edges from their own tiles
    (no ghost copies); a lattice off every tile multiple, against kernel 1."""
    nx, ny = 75, 41
    solid = np.zeros((ny, nx), np.uint8)
    if not periodic_y:
        solid[0] = solid[-1] = 1
    yy, xx = np.mgrid[0:ny, 0:nx]
    solid[(xx - 50) ** 2 + (yy - 20) ** 2 <= 30] = 1
    solid[(xx - 8) ** 2 + (yy - 31) ** 2 <= 12] = 1
    xi = media.uniform_xi(solid, -0.3)
    kw = dict(prec=prec, nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), periodic_y=periodic_y)
    if open_x:
        rho1, rho2 = media.drainage_densities(solid)
        kw.update(rho_in1=1.01, rho_out2=1.0)
    else:
        rho1, rho2 = media.droplet_densities(nx, ny, 70, 20, 9, solid=solid)
    a = mclbm.Lattice(solid, xi, kernel=1, **kw)
    b = mclbm.Lattice(solid, xi, kernel=4, tile_shape=tile_shape, **kw)
    a.init(rho1, rho2)
    b.init(rho1, rho2)
    a.step(1)
    b.step(1)
    scale = np.max(np.abs(a.populations()))
    assert np.max(np.abs(a.populations() - b.populations())) <= AGREE[prec][0] * scale
    a.step(199)
    b.step(199)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) <= AGREE[prec][1] * np.max(np.abs(fa))


@pytest.mark.parametrize("tile_shape", [0, 1])
@pytest.mark.parametrize("periodic_y,open_x", [(True, False), (False, True)])
def test_fluid_only_kernel_speckle_medium_fp32(periodic_y, open_x, tile_shape):
    """Isolated solid nodes scattered at random (30 %) leave fluid ring nodes
    whose fluid neighbours are neither own nor ring nodes: the tile must
    still stage the ring node's own populations, which its bounce-back and
    Set-3 treatment read.  Kernel 4 against the oracle on a lattice off every
    tile multiple."""
    nx, ny = 97, 50
    rng = np.random.default_rng(5)
    solid = (rng.random((ny, nx)) < 0.3).astype(np.uint8)
    if not periodic_y:
        solid[0] = solid[-1] = 1
    if open_x:
        solid[:, :2] = 0
        solid[:, -2:] = 0
        if not periodic_y:
            solid[0] = solid[-1] = 1
    xi = media.uniform_xi(solid, -0.3)
    kw = dict(nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), periodic_y=periodic_y)
    if open_x:
        rho1, rho2 = media.drainage_densities(solid)
        kw.update(rho_in1=1.01, rho_out2=1.0)
    else:
        rho1, rho2 = media.droplet_densities(nx, ny, 48, 25, 12, solid=solid)
    o = oracle.Oracle(solid, xi, **kw)
    o.init(rho1, rho2)
    g = mclbm.Lattice(solid, xi, prec="fp32", kernel=4, tile_shape=tile_shape, **kw)
    g.init(rho1, rho2)
    o.step(200)
    g.step(200)
    assert rel_err(g.populations(), o.f) < 2e-5


def test_fluid_only_readouts_and_kernel_switches():
    """Read-outs between fluid-only steps convert the layouts without loss,
    and switching kernels mid-run continues the same trajectory."""
    m = media.make_disk_medium(150, 70, 5, radius="uniform", r_lo=3.0, r_hi=6.0, porosity=0.7)
    xi = media.uniform_xi(m.solid, -0.3)
    rho1, rho2 = media.drainage_densities(m.solid)
    kw = dict(prec="fp32", nu1=nu_of_tau(1.7), nu2=nu_of_tau(0.62), rho_in1=1.01, rho_out2=1.0)
    a = mclbm.Lattice(m.solid, xi, kernel=4, **kw)
    b = mclbm.Lattice(m.solid, xi, kernel=4, **kw)
    a.init(rho1, rho2)
    b.init(rho1, rho2)
    a.step(100)
    for _ in range(10):
        b.step(10)
        b.diagnostics()
        b.density()
    assert np.array_equal(a.populations(), b.populations())
    assert a.diagnostics() == b.diagnostics()
    # kernel 4 -> 3 -> 4 against kernel 3 throughout
    c = mclbm.Lattice(m.solid, xi, kernel=3, **kw)
    c.init(rho1, rho2)
    c.step(100)
    mclbm.mclbm_set_flag(a.h, mclbm.MCLBM_FLAG_KERNEL, 3)
    a.step(50)
    c.step(50)
    mclbm.mclbm_set_flag(a.h, mclbm.MCLBM_FLAG_KERNEL, 4)
    a.step(50)
    c.step(50)
    fa, fc = a.populations(), c.populations()
    assert np.max(np.abs(fa - fc)) <= AGREE["fp32"][1] * np.max(np.abs(fc))


def test_fluid_only_kernel_paper_scale_medium():
    """The heterogeneous lognormal disk medium at 1024x512 (many tiles,
    mixed band sizes) against the dense tile kernel."""
    c = media.config_paper_scale(1024, 512, 1)
    kw = dict(prec="fp32", nu1=c["nu1"], nu2=c["nu2"], rho_in1=1.005, rho_out2=1.0)
    a = mclbm.Lattice(c["solid"], c["xi"], kernel=3, **kw)
    b = mclbm.Lattice(c["solid"], c["xi"], kernel=4, **kw)
    a.init(c["rho1"], c["rho2"])
    b.init(c["rho1"], c["rho2"])
    a.step(50)
    b.step(50)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb)) <= AGREE["fp32"][1] * np.max(np.abs(fa))
    assert a.diagnostics()["mass1"] == pytest.approx(b.diagnostics()["mass1"], rel=1e-6)
