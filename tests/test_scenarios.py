"""The paper-geometry generators against the values the paper prints for
them (no GPU, no oracle): Whalin's shoal (Sec. 4.2, Eq. 37, with the
ramp's sign read so that it rises from 0.4572 m to the 0.1524 m deep
shallow end the text gives), the conical island (Sec. 4.3) and the planar
beach (Sec. 4.1)."""
import math

import numpy as np

from paper_1611_05984_gb300 import scenarios as sc


def test_whalin_geometry():
    s = sc.whalin()
    assert (s.nx, s.ny) == (2000, 65) and s.dt == 0.001
    assert math.isclose(s.nx * s.dx, 35.0) and math.isclose(s.ny * s.dy, 6.096)
    x = (np.arange(s.nx) + 0.5) * s.dx
    y = (np.arange(s.ny) + 0.5) * s.dy
    depth = -s.z
    for j in (0, s.ny // 2, s.ny - 1):
        G = math.sqrt(y[j] * (6.096 - y[j]))
        x0, x1 = 10.67 - G, 18.29 - G
        flat, top = x < x0, x >= x1
        ramp = ~flat & ~top
        np.testing.assert_allclose(depth[j, flat], 0.4572, rtol=0, atol=1e-12)
        np.testing.assert_allclose(depth[j, top], 0.1524, rtol=0, atol=1e-12)
        np.testing.assert_allclose(depth[j, ramp], 0.4572 - (x[ramp] - x0) / 25.0, rtol=0, atol=1e-12)
    # the sine maker (a = 0.0075 m, T = 2 s) on the west, a 5 m sponge on
    # the east, walls north and south
    assert s.sides[sc.W].type == sc.SINE and s.sides[sc.W].comps[0][:2] == (0.0075, 2.0)
    assert s.sides[sc.E].type == sc.SPONGE and math.isclose(s.sides[sc.E].width * s.dx, 5.0, rel_tol=0.01)
    assert s.sides[sc.S].type == sc.SOLID and s.sides[sc.N].type == sc.SOLID


def test_conical_island_geometry():
    """Sec. 4.3: a 30 m x 30 m domain on 601 x 601 cells, dt = 0.005 s,
    0.32 m deep, a cone of 7.2 m base diameter and 1/4 side slope in the
    centre, sponges on the sides parallel to the soliton's crest (west and
    east), walls on the others, no friction, the soliton near the west."""
    s = sc.conical_island(0.09)
    assert (s.nx, s.ny) == (601, 601) and s.dt == 0.005 and s.friction == 0
    assert math.isclose(s.nx * s.dx, 30.0) and math.isclose(s.ny * s.dy, 30.0)
    x = (np.arange(s.nx) + 0.5) * s.dx
    r = np.hypot(x[None, :] - 15.0, x[:, None] - 15.0)
    depth = -s.z
    np.testing.assert_allclose(depth[r >= 3.6], 0.32, rtol=0, atol=1e-12)      # the floor beyond the 7.2 m base
    flank = (r < 3.6) & (depth > 0.32 - 0.625 + 1e-9)                          # below the cut top
    np.testing.assert_allclose(depth[flank], 0.32 - (3.6 - r[flank]) / 4.0, rtol=0, atol=1e-12)
    shore = r[np.abs(depth) < 0.01]
    assert abs(shore.mean() - 2.32) < 0.03                                      # 3.6 - 4 x 0.32
    assert s.sides[sc.W].type == sc.SPONGE and s.sides[sc.E].type == sc.SPONGE
    assert s.sides[sc.S].type == sc.SOLID and s.sides[sc.N].type == sc.SOLID
    (H, theta, x0, _), = s.solitons
    assert math.isclose(H, 0.09 * 0.32) and theta == 0.0 and x0 < 7.5


def test_planar_beach_geometry():
    """Sec. 4.1: a 1:19.85 beach, dx / d = 0.25 and dt sqrt(g/d) = 0.03
    (0.0625 and 0.0075 for H/d < 0.01), a tank one depth wide, a sponge on
    the west and walls elsewhere, quadratic friction f."""
    for H, dxd, dtd in ((0.28, 0.25, 0.03), (0.005, 0.0625, 0.0075)):
        s = sc.planar_beach_soliton(H_over_d=H, d=1.0, f=0.01)
        assert math.isclose(s.dx, dxd) and math.isclose(s.dt * math.sqrt(9.81), dtd)
        assert abs(s.ny * s.dy - 1.0) <= s.dy
        z = s.z[0]
        on_slope = z[:-1] > -1.0 + 1e-12          # both cells of the difference on the beach
        assert np.count_nonzero(on_slope) > 10
        np.testing.assert_allclose(np.diff(z)[on_slope], s.dx / 19.85, rtol=1e-9)
        assert s.sides[sc.W].type == sc.SPONGE and s.friction == 1 and s.fcoef == 0.01
        assert all(s.sides[k].type == sc.SOLID for k in (sc.E, sc.S, sc.N))
