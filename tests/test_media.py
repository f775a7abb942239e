"""Input generators: the layout of the U-obstacle channel that stands in
for the geometry of Sec. 4.1."""
import numpy as np

from paper_2111_08666_gb300 import media



def test_u_obstacle_channel_layout():
    """The Sec. 4.1 stand-in: walls, a U open towards the inlet with the
    droplet of component 1 inside it, and fluid region masks."""
    c = media.config_u_obstacle()
    solid, fluid = c["solid"], c["solid"] == 0
    assert c["solid"].shape == (200, 800)
    assert solid[:2].all() and solid[-2:].all()
    for k in ("cavity", "front", "behind"):
        assert (c[k] & fluid).sum() == c[k].sum() > 0  # regions are fluid
    # the cup is closed towards the outlet and open towards the inlet
    ys = np.nonzero(c["cavity"].any(axis=1))[0]
    xs = np.nonzero(c["cavity"].any(axis=0))[0]
    assert solid[ys, xs.max() + 1].all() and not solid[ys, xs.min() - 1].any()
    # the droplet: component 1 dominates a half disk of radius ~30 in the cup
    oil_in_cup = (c["rho1"] > c["rho2"]) & c["cavity"]
    assert abs(oil_in_cup.sum() - np.pi * 30 ** 2 / 2) < 0.05 * np.pi * 30 ** 2 / 2
    assert (c["rho1"][:, :5][fluid[:, :5]] == 1.0).all()


def test_block_medium_stand_in():
    """Block stand-in of Sec. 4.2: 10x10 blocks, porosity at the paper's
    0.8117, solid walls, block-free reservoirs, gaps between blocks."""
    m = media.make_block_medium()
    s = m.solid
    assert s.shape == (200, 400) and abs(m.porosity - 0.8117) < 0.002
    assert s[:2].all() and s[-2:].all()
    assert not s[2:-2, :10].any() and not s[2:-2, -10:].any()
    for x0, y0 in m.disks.astype(int):
        assert s[y0:y0 + 10, x0:x0 + 10].all()
        ring = s[max(y0 - 3, 0):y0 + 13, max(x0 - 3, 0):x0 + 13].sum()
        assert ring == 100  # nothing else within 3 nodes
    c = media.config_block_hysteresis(110.0)
    assert c["xi_value"] == 0.2 and c["xi"][s == 1].max() == np.float32(0.2)
