"""Host checks of the fluid-only layout (kernel 4), no GPU: the builder cuts
each band of rows into tiles of at most 32 columns and at most one fluid
node per compute thread, orders every tile's fluid nodes into slot blocks,
and writes per tile the work lists and the copy ranges that stage what the
tile reads.  The library's own self-check then verifies, against the
geometry, what the step kernel relies on: every fluid node sits in exactly
one block; every pull of an own or ring node (Sec. 2.1, half-way
bounce-back) finds its fluid source staged as a whole node of one copy at
its frame position, with the right global slot; every neighbour an own
node's force stencil reads (Eqs. 12-15) has a density or a virtual
density, and every fluid neighbour of a virtual-density node (Eqs. 16-17)
has a density; copies stay inside the stage and the population buffer and
do not overlap.  Sizes stay within the shared memory of the target CTAs
per SM (three for 12-row bands, two for 16-row bands)."""
import numpy as np
import pytest

from paper_2111_08666_gb300 import mclbm, media

GEO_OUTSIDE = 255
NT = {0: 256, 1: 384}                      # compute threads per CTA
SMEM_BUDGET = {0: 233472 // 3 - 1024, 1: 233472 // 2 - 1024}


def codes_of(solid: np.ndarray, periodic_x: bool = True, periodic_y: bool = False) -> np.ndarray:
    """Geometry codes over [-3, nx + 3) x [-3, ny + 3): 0 fluid, 1 solid,
    ghosts as copies of the opposite edge where periodic, else outside."""
    ny, nx = solid.shape
    c = np.full((ny + 6, nx + 6), GEO_OUTSIDE, np.uint8)
    core = np.where(solid > 0, 1, 0).astype(np.uint8)
    c[3:ny + 3, 3:nx + 3] = core
    if periodic_x:
        c[3:ny + 3, 0:3] = core[:, nx - 3:]
        c[3:ny + 3, nx + 3:] = core[:, :3]
    if periodic_y:
        c[0:3, :] = c[ny:ny + 3, :]
        c[ny + 3:, :] = c[3:6, :]
    return c


def _disk(nx, ny, seed, porosity=0.6):
    return media.make_disk_medium(nx, ny, seed, porosity=porosity).solid


def _geometries():
    rng = np.random.default_rng(5)
    channel = np.zeros((45, 160), np.uint8)
    channel[:2] = 1
    channel[-2:] = 1
    channel[15:30, 40:48] = 1
    channel[5:12, 100:130] = 1
    speckle = (rng.random((50, 97)) < 0.3).astype(np.uint8)
    one = np.ones((20, 40), np.uint8)
    one[10, 17] = 0
    return {
        "disk 256x128": (_disk(256, 128, 3), dict()),
        "fluid 101x37 (ragged)": (np.zeros((37, 101), np.uint8), dict()),
        "fluid 101x37 periodic y": (np.zeros((37, 101), np.uint8), dict(periodic_y=True)),
        "channel 160x45 periodic y": (channel, dict(periodic_y=True)),
        "speckle 97x50": (speckle, dict(periodic_y=True)),
        "no fluid 64x32": (np.ones((32, 64), np.uint8), dict()),
        "one fluid node": (one, dict()),
        "disk 200x96 open x": (_disk(200, 96, 7), dict(periodic_x=False, open_x=True)),
        "narrow 5x40": (np.zeros((40, 5), np.uint8), dict(periodic_y=True)),
    }


GEOMETRIES = _geometries()


@pytest.mark.parametrize("name", list(GEOMETRIES))
@pytest.mark.parametrize("shape", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp16dev"])
def test_layout_stages_every_read(name, shape, prec):
    solid, kw = GEOMETRIES[name]
    open_x = kw.get("open_x", False)
    codes = codes_of(solid, kw.get("periodic_x", True), kw.get("periodic_y", False))
    r = mclbm.mclbm_fluid_layout_check(codes, prec, shape, open_x)
    assert r["check"] == 0, r
    fluid = int((solid == 0).sum())
    assert r["slots"] >= fluid
    # one fluid node per compute thread (the own block adds at most one
    # padding slot to each of its nine bands)
    assert r["max_own"] <= NT[shape] + 9
    assert r["tiles"] >= -(-fluid // NT[shape])
    assert r["smem_bytes"] <= SMEM_BUDGET[shape]
    assert 1 <= r["attempts"] <= 8


@pytest.mark.parametrize("shape", [0, 1])
def test_layout_of_the_2048x1024_medium(shape):
    """The heterogeneous disk medium of the throughput workload: within the
    budget of three (two) CTAs per SM, in a few attempts."""
    c = media.config_paper_scale(2048, 1024, 99)
    r = mclbm.mclbm_fluid_layout_check(codes_of(c["solid"]), "fp32", shape)
    assert r["check"] == 0, r
    assert r["smem_bytes"] <= SMEM_BUDGET[shape]
    assert r["attempts"] <= 4
    fluid = int((c["solid"] == 0).sum())
    # tiles hold 0.8-1 of a CTA's threads on average
    assert fluid / r["tiles"] > 0.8 * NT[shape] * (0.9 if shape == 0 else 0.75)


def test_tiles_are_narrower_where_the_medium_is_open():
    """A fully fluid band holds at most NT fluid nodes per tile: 12-row
    bands of an open lattice need at least ceil(nx / 21) tiles per band,
    where a 32-column tiling would use ceil(nx / 32)."""
    nx, ny = 320, 24
    r = mclbm.mclbm_fluid_layout_check(codes_of(np.zeros((ny, nx), np.uint8), periodic_y=True), "fp32", 0)
    assert r["check"] == 0
    assert r["tiles"] >= 2 * -(-nx // 21)
    sparse = np.ones((ny, nx), np.uint8)
    sparse[:, ::4] = 0  # a quarter fluid: 32-column tiles hold 96 fluid nodes
    r = mclbm.mclbm_fluid_layout_check(codes_of(sparse, periodic_y=True), "fp32", 0)
    assert r["check"] == 0
    assert r["tiles"] == 2 * (nx // 32)


def test_layout_check_rejects_bad_arguments():
    codes = codes_of(np.zeros((16, 16), np.uint8))
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_fluid_layout_check(codes, "fp64", 0)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_fluid_layout_check(codes, "fp32", 2)
    with pytest.raises(ValueError):
        mclbm.mclbm_fluid_layout_check(np.zeros((5, 5), np.uint8))


def _random_geometry(rng):
    """A ragged lattice with one of three solid patterns: speckle (isolated
    solids), blobs (clustered solids) or stripes with gaps, at a random
    porosity, with or without walls."""
    ny, nx = int(rng.integers(5, 70)), int(rng.integers(5, 140))
    kind = rng.integers(3)
    phi = rng.uniform(0.2, 0.95)
    if kind == 0:
        solid = (rng.random((ny, nx)) > phi).astype(np.uint8)
    elif kind == 1:
        solid = np.zeros((ny, nx), np.uint8)
        yy, xx = np.mgrid[0:ny, 0:nx]
        for _ in range(int(rng.integers(1, 12))):
            cy, cx, r = rng.uniform(0, ny), rng.uniform(0, nx), rng.uniform(1, 8)
            solid[(yy - cy) ** 2 + (xx - cx) ** 2 < r * r] = 1
    else:
        solid = np.zeros((ny, nx), np.uint8)
        for x in range(int(rng.integers(0, 4)), nx, int(rng.integers(3, 9))):
            solid[:, x] = 1
            solid[rng.integers(0, ny):, x] = 0
    walls = bool(rng.integers(2)) and ny > 4
    if walls:
        solid[:2] = 1
        solid[-2:] = 1
    return solid, dict(periodic_y=not walls, open_x=bool(rng.integers(2)))


@pytest.mark.parametrize("seed", range(24))
def test_layout_of_random_geometries(seed):
    """Seeded random geometries (sizes, patterns, porosities, boundary
    modes, both band heights and both storage widths): every invariant of
    the self-check holds and every fluid node sits in one block."""
    rng = np.random.default_rng(1000 + seed)
    solid, kw = _random_geometry(rng)
    shape = int(rng.integers(2))
    prec = ("fp32", "fp16dev")[int(rng.integers(2))]
    codes = codes_of(solid, periodic_x=not kw["open_x"], periodic_y=kw["periodic_y"])
    r = mclbm.mclbm_fluid_layout_check(codes, prec, shape, kw["open_x"])
    assert r["check"] == 0, (seed, solid.shape, kw, shape, prec, r)
    fluid = int((solid == 0).sum())
    assert r["slots"] >= fluid
    assert r["max_own"] <= NT[shape] + 9
    assert r["smem_bytes"] <= SMEM_BUDGET[shape]
