"""Seeded synthetic inputs: porous media, initial density fields, wettability maps.

This module is the only code shared by the CUDA path, the CPU oracle and the
benchmark.  It holds none of the lattice Boltzmann arithmetic: it draws
geometries and initial fields, nothing else.

The paper's own porous medium (400x200 blocks of 10x10, porosity 81.17 %,
Sec. 4.2.1) comes from another publication and is not available here, so
disk packings of the sizes, porosities and radius laws of the workloads stand
in for it.  The layout of the stand-in follows Sec. 4.2.1: solid walls at the
top and bottom, ten disk-free columns at each end as fluid reservoirs, and
five columns of the non-wetting fluid (component 1, oil) at the inlet.

Arrays are row-major ``[y][x]``; x is the flow direction, the inlet is x=0
and the outlet x=nx-1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Densities of the two phases after separation at G=3.5 (Sec. 3.2): the
# majority component sits at 1, the dissolved minority at 0.027.
RHO_MAJOR = 1.0
RHO_MINOR = 0.027


@dataclass
class Medium:
    solid: np.ndarray      # uint8 [ny][nx], 1 = solid
    disks: np.ndarray      # float64 [n][3] (cx, cy, r)
    porosity: float        # fluid nodes / all nodes


def _uniform_radius(lo: float, hi: float):
    def draw(rng: np.random.Generator, x: float, nx: int) -> float:
        return float(rng.uniform(lo, hi))
    return draw


def _lognormal_radius(mean: float, sigma_log: float, fine_from: float | None,
                      fine_scale: float, r_min: float):
    mu_log = math.log(mean) - 0.5 * sigma_log * sigma_log

    def draw(rng: np.random.Generator, x: float, nx: int) -> float:
        r = float(rng.lognormal(mu_log, sigma_log))
        if fine_from is not None and x >= fine_from * nx:
            r *= fine_scale
        return max(r, r_min)
    return draw


def make_disk_medium(nx: int, ny: int, seed: int, *, radius: str = "uniform",
                     r_lo: float = 4.0, r_hi: float = 8.0, r_mean: float = 10.0,
                     sigma_log: float = 0.4, heterogeneous: bool = False,
                     porosity: float = 0.65, wall_rows: int = 2,
                     reservoir: int = 10, min_gap: float = 2.0,
                     max_failures: int = 100_000) -> Medium:
    """Random sequential addition of non-overlapping disks.

    A centre is drawn uniformly in the disk-allowed box and a radius from the
    chosen law; the disk is rejected when it comes closer than ``min_gap``
    nodes to another disk, to a wall or to a reservoir.  Node (x, y) is solid
    when (x-cx)^2 + (y-cy)^2 <= r^2.  Placement stops once the porosity is at
    or below the target, or after ``max_failures`` consecutive rejections.

    ``radius="lognormal"`` draws radii with arithmetic mean ``r_mean`` and
    log-standard-deviation ``sigma_log``; with ``heterogeneous=True`` the
    radii in the downstream half (x >= nx/2) are halved, giving a coarse and
    a fine region.
    """
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    if wall_rows > 0:
        solid[:wall_rows, :] = 1
        solid[ny - wall_rows:, :] = 1
    if radius == "uniform":
        draw = _uniform_radius(r_lo, r_hi)
    elif radius == "lognormal":
        draw = _lognormal_radius(r_mean, sigma_log, 0.5 if heterogeneous else None,
                                 0.5, 1.5)
    else:
        raise ValueError(radius)

    x_lo, x_hi = float(reservoir), float(nx - reservoir - 1)
    y_lo, y_hi = float(wall_rows), float(ny - wall_rows - 1)
    centres = np.zeros((0, 3))
    # cell list so that the overlap test only looks at nearby disks
    cell = 24.0
    grid: dict[tuple[int, int], list[int]] = {}
    disks: list[tuple[float, float, float]] = []
    failures = 0
    n_all = nx * ny
    n_solid = int(solid.sum())
    yy, xx = np.mgrid[0:ny, 0:nx]
    r_max_seen = 0.0
    while n_solid / n_all < 1.0 - porosity and failures < max_failures:
        cx = float(rng.uniform(x_lo, x_hi))
        cy = float(rng.uniform(y_lo, y_hi))
        r = draw(rng, cx, nx)
        ok = (cx - r - min_gap >= x_lo and cx + r + min_gap <= x_hi and
              cy - r - min_gap >= y_lo and cy + r + min_gap <= y_hi)
        if ok:
            reach = r + min_gap + r_max_seen
            gx0, gx1 = int((cx - reach) // cell), int((cx + reach) // cell)
            gy0, gy1 = int((cy - reach) // cell), int((cy + reach) // cell)
            for gx in range(gx0, gx1 + 1):
                for gy in range(gy0, gy1 + 1):
                    for k in grid.get((gx, gy), ()):
                        ox, oy, orad = disks[k]
                        if math.hypot(cx - ox, cy - oy) - r - orad < min_gap:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
        if not ok:
            failures += 1
            continue
        failures = 0
        k = len(disks)
        disks.append((cx, cy, r))
        grid.setdefault((int(cx // cell), int(cy // cell)), []).append(k)
        r_max_seen = max(r_max_seen, r)
        x0, x1 = max(int(math.floor(cx - r)), 0), min(int(math.ceil(cx + r)), nx - 1)
        y0, y1 = max(int(math.floor(cy - r)), 0), min(int(math.ceil(cy + r)), ny - 1)
        sub_x = xx[y0:y1 + 1, x0:x1 + 1]
        sub_y = yy[y0:y1 + 1, x0:x1 + 1]
        inside = (sub_x - cx) ** 2 + (sub_y - cy) ** 2 <= r * r
        block = solid[y0:y1 + 1, x0:x1 + 1]
        n_solid += int((inside & (block == 0)).sum())
        block[inside] = 1
    if disks:
        centres = np.asarray(disks, dtype=np.float64)
    return Medium(solid=solid, disks=centres, porosity=1.0 - n_solid / n_all)


def drainage_densities(solid: np.ndarray, oil_columns: int = 5):
    """Initial state of primary drainage (Sec. 4.2.1): oil (component 1) at
    (1, 0.027) in the first ``oil_columns`` columns, water (component 2) at
    the reversed densities elsewhere.  Solid nodes carry zeros."""
    ny, nx = solid.shape
    rho1 = np.full((ny, nx), RHO_MINOR)
    rho2 = np.full((ny, nx), RHO_MAJOR)
    rho1[:, :oil_columns] = RHO_MAJOR
    rho2[:, :oil_columns] = RHO_MINOR
    fluid = solid == 0
    return rho1 * fluid, rho2 * fluid


def droplet_densities(nx: int, ny: int, xc: float, yc: float, r0: float,
                      width: float = 5.0, rho_hi: float = RHO_MAJOR,
                      rho_lo: float = RHO_MINOR, solid: np.ndarray | None = None):
    """Diffuse droplet of component 1 in component 2, the tanh profile of
    Eq. 29 (interface width W, centre (xc, yc), radius r0)."""
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.sqrt((xx - xc) ** 2 + (yy - yc) ** 2)
    t = np.tanh(2.0 * (d - r0) / width)
    rho1 = 0.5 * (rho_hi + rho_lo) - 0.5 * (rho_hi - rho_lo) * t
    rho2 = 0.5 * (rho_lo + rho_hi) - 0.5 * (rho_lo - rho_hi) * t
    if solid is not None:
        rho1 = rho1 * (solid == 0)
        rho2 = rho2 * (solid == 0)
    return rho1, rho2


def layered_densities(ny: int, nx: int, y_split: float, width: float = 5.0,
                      rho_hi: float = RHO_MAJOR, rho_lo: float = RHO_MINOR,
                      solid: np.ndarray | None = None):
    """Flat diffuse interface: component 1 below ``y_split``, component 2
    above, with the tanh profile of Eq. 29 taken along y."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    t = np.tanh(2.0 * (y - y_split) / width)
    rho1 = 0.5 * (rho_hi + rho_lo) - 0.5 * (rho_hi - rho_lo) * t
    rho2 = 0.5 * (rho_lo + rho_hi) - 0.5 * (rho_lo - rho_hi) * t
    if solid is not None:
        rho1 = rho1 * (solid == 0)
        rho2 = rho2 * (solid == 0)
    return rho1, rho2


def theta_to_xi(theta_deg: float) -> float:
    """Wettability parameter for a contact angle, by inverting the cubic fit
    of Sec. 3.3, theta = 47.5487 xi^3 - 13.9067 xi^2 + 92.0987 xi + 90.8074.
    The cubic is strictly increasing (its derivative has no real root), so
    bisection finds the unique root."""
    def theta(xi: float) -> float:
        return ((47.5487 * xi - 13.9067) * xi + 92.0987) * xi + 90.8074
    lo, hi = -2.0, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if theta(mid) < theta_deg:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def uniform_xi(solid: np.ndarray, xi: float) -> np.ndarray:
    """Per-site wettability map with one value on every solid node."""
    return np.where(solid != 0, np.float32(xi), np.float32(0.0)).astype(np.float32)


# --- the workloads -----------------------------------------------------------

def config_small_fp64():
    """128x64 disk medium, radii U[4, 8], seed 0, porosity ~0.65, neutral
    wetting (xi = 0), viscosity ratio 1 (tau = 1 for both components)."""
    m = make_disk_medium(128, 64, 0, radius="uniform", r_lo=4.0, r_hi=8.0,
                         porosity=0.65)
    rho1, rho2 = drainage_densities(m.solid)
    return dict(name="disk128x64_fp64", nx=128, ny=64, solid=m.solid,
                xi=uniform_xi(m.solid, 0.0), rho1=rho1, rho2=rho2,
                nu1=1.0 / 6.0, nu2=1.0 / 6.0, g=3.5, rho_in1=1.01, rho_out2=1.0,
                porosity=m.porosity)


def config_paper_scale(nx: int = 1024, ny: int = 512, seed: int = 1):
    """Heterogeneous lognormal disk medium (arithmetic mean radius 10,
    sigma_log 0.4, radii halved for x >= nx/2), porosity ~0.6, water-wet
    theta = 50 deg, viscosity ratio 10 (tau1 = 1.7, tau2 = 0.62)."""
    m = make_disk_medium(nx, ny, seed, radius="lognormal", r_mean=10.0,
                         sigma_log=0.4, heterogeneous=True, porosity=0.6)
    rho1, rho2 = drainage_densities(m.solid)
    xi = theta_to_xi(50.0)
    return dict(name=f"hetero_disk{nx}x{ny}_fp32", nx=nx, ny=ny, solid=m.solid,
                xi=uniform_xi(m.solid, xi), rho1=rho1, rho2=rho2,
                nu1=(1.7 - 0.5) / 3.0, nu2=(0.62 - 0.5) / 3.0, g=3.5,
                rho_in1=1.0, rho_out2=1.0, porosity=m.porosity)


def config_batch(k: int):
    """Case k (0..23) of the batched workload: disk medium of seed 10 + k,
    size drawn from {256x256, 512x256, 512x512, 1024x256, 1024x512},
    contact angle 30 + 120 k / 23 deg, viscosity ratio cycling 1, 10, 50
    (tau2 = 0.62, or 0.56 at M = 50), primary drainage set-up."""
    sizes = [(256, 256), (512, 256), (512, 512), (1024, 256), (1024, 512)]
    nx, ny = sizes[int(np.random.default_rng(k).integers(len(sizes)))]
    m = make_disk_medium(nx, ny, 10 + k, radius="lognormal", r_mean=10.0, sigma_log=0.4,
                         porosity=0.6)
    theta = 30.0 + 120.0 * k / 23.0
    taus = [(1.0, 1.0), (1.7, 0.62), (3.5, 0.56)][k % 3]
    rho1, rho2 = drainage_densities(m.solid)
    return dict(name=f"batch{k}_{nx}x{ny}", nx=nx, ny=ny, solid=m.solid,
                xi=uniform_xi(m.solid, theta_to_xi(theta)), rho1=rho1, rho2=rho2,
                nu1=(taus[0] - 0.5) / 3.0, nu2=(taus[1] - 0.5) / 3.0, g_coh=3.5,
                rho_in1=1.005, rho_out2=1.0, porosity=m.porosity, theta=theta)


def config_u_obstacle(nx: int = 800, ny: int = 200, arm: int = 10, r_drop: float = 30.0):
    """Channel with a U-shaped wall (Sec. 4.1), a stand-in with dimensions of
    our own: the paper gives the 800x200 channel, the droplet radius 30 and
    the physics, not the obstacle's size.

    Walls: rows 0-1 and ny-2..ny-1.  The U spans x in [nx/4, nx/4 + 80) and
    the middle half of the channel (y in [ny/4, 3 ny/4)), its opening facing
    the inlet and its closed side (thickness ``arm``) the outlet, so that the
    invading component flows through the passages above and below while the
    water inside the cup has nowhere to go.  A semicircular droplet of
    component 1 (radius ``r_drop``) sits on the inner face of the closed
    side; component 1 also fills the first 5 columns, component 2 the rest.
    Physics of Sec. 4.1: tau1 = 3.5, tau2 = 0.62 (M = 25), xi = -0.4,
    rho_in1 = 1.01, rho_out2 = 1.  ``cavity`` marks the inside of the cup."""
    solid = np.zeros((ny, nx), np.uint8)
    solid[:2] = 1
    solid[-2:] = 1
    x0, x1 = nx // 4, nx // 4 + 80
    y0, y1 = ny // 4, 3 * ny // 4
    solid[y0:y1, x1 - arm:x1] = 1      # closed side
    solid[y0:y0 + arm, x0:x1] = 1      # lower arm
    solid[y1 - arm:y1, x0:x1] = 1      # upper arm
    cavity = np.zeros((ny, nx), bool)
    cavity[y0 + arm:y1 - arm, x0:x1 - arm] = True
    front = np.zeros((ny, nx), bool)
    front[y0:y1, x0 - 50:x0] = True
    behind = np.zeros((ny, nx), bool)
    behind[y0 - 10:y1 + 10, x1:x1 + 60] = True
    rho1, rho2 = drainage_densities(solid)
    # the droplet: tanh profile of Eq. 29 centred on the inner face
    d1, d2 = droplet_densities(nx, ny, x1 - arm, 0.5 * (y0 + y1), r_drop, solid=solid)
    inner = np.zeros((ny, nx), bool)
    inner[:, : x1 - arm] = True
    drop = inner & (d1 > rho1)
    rho1 = np.where(drop, d1, rho1)
    rho2 = np.where(drop, d2, rho2)
    return dict(name=f"u_obstacle{nx}x{ny}", nx=nx, ny=ny, solid=solid, cavity=cavity, front=front, behind=behind,
                xi=uniform_xi(solid, -0.4), rho1=rho1 * (solid == 0), rho2=rho2 * (solid == 0),
                nu1=(3.5 - 0.5) / 3.0, nu2=(0.62 - 0.5) / 3.0, g=3.5, rho_in1=1.01, rho_out2=1.0)


def make_block_medium(nx: int = 400, ny: int = 200, seed: int = 24, *, block: int = 10,
                      porosity: float = 0.8117, gap: int = 3, wall_rows: int = 2,
                      reservoir: int = 10, max_failures: int = 100_000) -> Medium:
    """Random sequential addition of square solid blocks (side ``block``),
    a stand-in for the block medium of Sec. 4.2 (400x200, 10x10 blocks,
    porosity 0.8117, solid walls, block-free reservoirs of 10 columns at each
    end; the paper takes its geometry from its ref. [24], which is not
    available).  A corner is drawn uniformly on the integer grid of the
    allowed box; the block is rejected when it comes closer than ``gap``
    nodes to another block, a wall or a reservoir.  Placement stops once the
    porosity (all nodes) is at or below the target, or after
    ``max_failures`` consecutive rejections."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[:wall_rows, :] = 1
    solid[ny - wall_rows:, :] = 1
    # occupied: blocks grown by the gap, so that a new block must avoid it
    keep_out = np.zeros((ny, nx), bool)
    keep_out[: wall_rows + gap] = True
    keep_out[ny - wall_rows - gap:] = True
    keep_out[:, : reservoir + gap] = True
    keep_out[:, nx - reservoir - gap:] = True
    corners = []
    failures = 0
    n_all = nx * ny
    while 1.0 - solid.sum() / n_all > porosity and failures < max_failures:
        x0 = int(rng.integers(0, nx - block + 1))
        y0 = int(rng.integers(0, ny - block + 1))
        if keep_out[y0:y0 + block, x0:x0 + block].any():
            failures += 1
            continue
        failures = 0
        corners.append((x0, y0))
        solid[y0:y0 + block, x0:x0 + block] = 1
        keep_out[max(y0 - gap, 0):y0 + block + gap, max(x0 - gap, 0):x0 + block + gap] = True
    return Medium(solid=solid, disks=np.asarray(corners, dtype=np.float64).reshape(-1, 2),
                  porosity=1.0 - solid.sum() / n_all)


# contact angle -> xi as Sec. 4.2 states them (22 deg: -0.55, 50 deg: -0.4,
# 110 deg: 0.2)
PAPER_XI = {22.0: -0.55, 50.0: -0.4, 110.0: 0.2}


def config_block_hysteresis(theta: float, seed: int = 24):
    """The drainage/imbibition workload of Sec. 4.2 on the block stand-in:
    viscosity ratio 25 (tau1 = 3.5, tau2 = 0.62), contact angle ``theta``
    (22, 50 or 110 deg, with the paper's xi for each), five oil layers at the
    inlet, equal boundary densities to start."""
    m = make_block_medium(seed=seed)
    rho1, rho2 = drainage_densities(m.solid)
    xi = PAPER_XI.get(float(theta), theta_to_xi(theta))
    return dict(name=f"block400x200_theta{theta:g}", nx=400, ny=200, solid=m.solid,
                xi=uniform_xi(m.solid, xi), xi_value=xi, rho1=rho1, rho2=rho2,
                nu1=(3.5 - 0.5) / 3.0, nu2=(0.62 - 0.5) / 3.0, g=3.5, rho_in1=1.0, rho_out2=1.0,
                porosity=m.porosity, theta=theta)
