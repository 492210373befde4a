"""Pins of the render oracle (the CPU restatement of the headless renderer)
against closed forms and invariants, computed here in FP64:

* Fresnel reflectance: the unpolarised Fresnel equations for air -> water
  (R = ((n - 1)/(n + 1))^2 at normal incidence, 1 at grazing incidence);
* colormaps: their control points and linearity between them;
* a flat lake seen from straight above: reflection of the zenith colour with
  the normal-incidence R, refraction of the bed colour weighted by
  1 / (1 + absorb h), by formula;
* flat land under a sun straight above is the bare terrain colour, and
  under a sun 60 degrees off the vertical the terrain colour times 0.675;
* grid lines where x / spacing crosses an integer;
* speed = |(P, Q)| / h, with h at least h_min;
* Lambert's law clamped at zero on land facing away from the sun;
* mirror symmetry: a state mirrored in x, seen and lit from the mirrored
  directions, renders as the mirrored image, byte for byte.
"""
import math

import numpy as np
import pytest

N2 = 1.333
SKY_ZENITH = np.array([0.250, 0.450, 0.800])
WATER = np.array([0.020, 0.150, 0.200])
TERRAIN0 = np.array([0.780, 0.700, 0.500])     # the terrain map at t = 0


def _fresnel64(cos_i):
    sin_t = math.sqrt(1 - cos_i ** 2) / N2
    cos_t = math.sqrt(1 - sin_t ** 2)
    rs = (cos_i - N2 * cos_t) / (cos_i + N2 * cos_t)
    rp = (N2 * cos_i - cos_t) / (N2 * cos_i + cos_t)
    return 0.5 * (rs * rs + rp * rp)


def _bytes(rgb):
    return np.array([int(min(max(c, 0.0), 1.0) * 255 + 0.5) for c in rgb])


def test_fresnel_closed_forms(oracle_mod):
    assert abs(oracle_mod.fresnel(1.0) - ((N2 - 1) / (N2 + 1)) ** 2) <= 1e-7
    assert abs(oracle_mod.fresnel(0.0) - 1.0) <= 1e-7
    prev = 2.0
    for c in np.linspace(0.0, 1.0, 41):
        r = oracle_mod.fresnel(float(c))
        assert abs(r - _fresnel64(c)) <= 2e-6
        assert r <= prev + 1e-7            # reflectance falls as the incidence steepens
        prev = r


def test_colormap_control_points_and_linearity(oracle_mod):
    for which in range(3):
        pts = [oracle_mod.colormap(which, k / 4) for k in range(5)]
        for k in range(4):
            mid = oracle_mod.colormap(which, (k + 0.5) / 4)
            np.testing.assert_allclose(mid, 0.5 * (pts[k] + pts[k + 1]), atol=1e-6)
        np.testing.assert_array_equal(oracle_mod.colormap(which, -3.0), pts[0])
        np.testing.assert_array_equal(oracle_mod.colormap(which, 7.0), pts[4])
    np.testing.assert_allclose(oracle_mod.colormap(2, 0.0), TERRAIN0, atol=1e-7)
    # five control points at t = 0, 1/4, ..., 1: the slope is constant inside
    # each quarter and changes at every inner control point
    for which in range(3):
        slope = [(oracle_mod.colormap(which, (k + 0.75) / 4) - oracle_mod.colormap(which, (k + 0.25) / 4)) * 8
                 for k in range(4)]
        for k in range(4):
            inner = (oracle_mod.colormap(which, (k + 0.5) / 4) - oracle_mod.colormap(which, (k + 0.25) / 4)) * 16
            np.testing.assert_allclose(inner, slope[k], atol=1e-4)
        for k in range(3):
            assert np.max(np.abs(slope[k + 1] - slope[k])) > 0.05


def test_flat_lake_from_above(oracle_mod):
    h, absorb = 2.0, 0.5
    w = np.zeros((6, 7))
    B = np.full((6, 7), -h)
    p = oracle_mod.render_params("fresnel", zmin=-h, zmax=1.0, absorb=absorb, view=(0.0, 0.0, -1.0))
    img = oracle_mod.render(w, w, w, B, 1.0, 1.0, 0.0, p)
    R = ((N2 - 1) / (N2 + 1)) ** 2
    refr = WATER + (TERRAIN0 - WATER) / (1 + absorb * h)   # the bed sits at zmin
    want = _bytes(R * SKY_ZENITH + (1 - R) * refr)
    assert np.all(np.abs(img[..., :3].astype(int) - want) <= 1)
    assert np.all(img[..., 3] == 255)
    assert np.all(img == img[0, 0])                          # uniform


def test_flat_land_hillshade(oracle_mod):
    z = np.full((5, 5), 0.5)
    w = z.copy()                                             # dry: w = bed
    p = oracle_mod.render_params("eta", zmin=0.5, zmax=1.5, sun=(0.0, 0.0, 1.0))
    img = oracle_mod.render(w, 0 * w, 0 * w, z, 1.0, 1.0, 0.0, p)
    assert np.all(np.abs(img[..., :3].astype(int) - _bytes(TERRAIN0)) <= 1)
    p = oracle_mod.render_params("eta", zmin=0.5, zmax=1.5, sun=(math.sin(math.pi / 3), 0.0, 0.5))
    img = oracle_mod.render(w, 0 * w, 0 * w, z, 1.0, 1.0, 0.0, p)
    assert np.all(np.abs(img[..., :3].astype(int) - _bytes(TERRAIN0 * (0.35 + 0.65 * 0.5))) <= 1)
    # Lambert's law clamps at zero: land rising steeply towards a low sun
    # faces away from it and keeps the ambient 0.35 of its terrain colour
    zs = np.tile(0.5 + 0.002 * np.arange(5.0), (5, 1))
    p = oracle_mod.render_params("eta", zmin=0.5, zmax=1.5, exaggeration=1000.0,
                                 sun=(math.sin(math.radians(80)), 0.0, math.cos(math.radians(80))))
    img = oracle_mod.render(zs, 0 * zs, 0 * zs, zs, 1.0, 1.0, 0.0, p)
    t = (zs[2, 2] - 0.5) / 1.0
    want = _bytes(oracle_mod.colormap(2, t).astype(np.float64) * 0.35)
    assert np.all(np.abs(img[2, 2, :3].astype(int) - want) <= 1)


def test_grid_lines(oracle_mod):
    nx, ny, dx = 40, 3, 0.5
    w = np.zeros((ny, nx))
    B = np.full((ny, nx), -1.0)
    base = oracle_mod.render(w, w, w, B, dx, 0.3, 0.0, oracle_mod.render_params("eta"))
    img = oracle_mod.render(w, w, w, B, dx, 0.3, 0.0, oracle_mod.render_params("eta", grid=2.0))
    darker = np.where(np.any(img[1, :, :3] != base[1, :, :3], axis=-1))[0]
    # x = (i + 1) dx crosses a multiple of 2 m for i = 3, 7, 11, ...
    np.testing.assert_array_equal(darker, np.arange(3, nx, 4))
    # and the rows: y = (j + 1) dy crosses a multiple of 1.5 m for j = 4, 9, 14, ...
    wt, Bt = np.zeros((nx, 3)), np.full((nx, 3), -1.0)
    base = oracle_mod.render(wt, wt, wt, Bt, 0.7, 0.3, 0.0, oracle_mod.render_params("eta"))
    img = oracle_mod.render(wt, wt, wt, Bt, 0.7, 0.3, 0.0, oracle_mod.render_params("eta", grid=1.5))
    darker = np.where(np.any(img[:, 1, :3] != base[:, 1, :3], axis=-1))[0]
    np.testing.assert_array_equal(darker, np.arange(4, nx, 5))


def test_speed_and_velocity_components(oracle_mod):
    h = 2.0
    B = np.full((3, 3), -h)
    w = np.zeros((3, 3))
    P = np.full((3, 3), 3.0 * h)
    Q = np.full((3, 3), 4.0 * h)
    for mode, val, m in (("speed", 5.0, 1), ("u", 3.0, 0), ("v", 4.0, 0)):
        p = oracle_mod.render_params(mode, vmin=0.0, vmax=10.0)
        img = oracle_mod.render(w, P, Q, B, 1.0, 1.0, 0.0, p)
        want = _bytes(oracle_mod.colormap(m, val / 10.0))
        np.testing.assert_array_equal(img[1, 1, :3], want)
    # a film thinner than h_min (but wet) shows its velocity over h_min:
    # P = 0.04 on 4 mm of water reads u = 2 (not 10)
    Bf = np.full((3, 3), -0.004)
    p = oracle_mod.render_params("u", vmin=0.0, vmax=10.0, dry_h=1e-3, h_min=0.02)
    img = oracle_mod.render(w, np.full((3, 3), 0.04), 0 * w, Bf, 1.0, 1.0, 0.0, p)
    np.testing.assert_array_equal(img[1, 1, :3], _bytes(oracle_mod.colormap(0, 0.2)))


@pytest.mark.parametrize("mode", ["fresnel", "eta", "v", "speed"])
def test_mirror_symmetry(oracle_mod, mode):
    rng = np.random.default_rng(3)
    ny, nx = 9, 12
    B = -1.0 + 1.2 * rng.random((ny, nx))
    w = np.maximum(B, 0.05 * rng.standard_normal((ny, nx)))
    P = 0.3 * rng.standard_normal((ny, nx))
    Q = 0.3 * rng.standard_normal((ny, nx))
    args = dict(vmin=-0.5, vmax=0.5, zmin=-1.0, zmax=0.5, grid=0.0, exaggeration=4.0)
    a = oracle_mod.render(w, P, Q, B, 1.0, 1.0, 0.0,
                          oracle_mod.render_params(mode, view=(0.4, 0.2, -1.0), sun=(0.5, 0.3, 1.0), **args))
    b = oracle_mod.render(w[:, ::-1], -P[:, ::-1], Q[:, ::-1], B[:, ::-1], 1.0, 1.0, 0.0,
                          oracle_mod.render_params(mode, view=(-0.4, 0.2, -1.0), sun=(-0.5, 0.3, 1.0), **args))
    np.testing.assert_array_equal(a, b[:, ::-1])


def test_tilted_plane_oblique_view(oracle_mod):
    """A plane water surface eta = s x seen along (0.6, 0, -0.8): the
    surface normal (-s, 0, 1)/sqrt(1 + s^2) gives cos i = (0.6 s + 0.8) /
    sqrt(1 + s^2) and the reflected ray's height -0.8 + 2 cos_i / sqrt(1 +
    s^2); the interior pixels follow by formula (the edges use one-sided
    differences of the same plane)."""
    nx, ny, dx, s, d = 12, 5, 0.1, 0.5, 3.0
    x = (np.arange(nx) + 0.5) * dx
    w = np.tile(s * x, (ny, 1))
    B = np.full((ny, nx), -d)
    p = oracle_mod.render_params("fresnel", zmin=-d, zmax=1.0, absorb=0.5, view=(0.6, 0.0, -0.8))
    img = oracle_mod.render(w, 0 * w, 0 * w, B, dx, dx, 0.0, p)
    nz = 1 / math.sqrt(1 + s * s)
    cos_i = (0.6 * s + 0.8) * nz
    R = _fresnel64(cos_i)
    rz = -0.8 + 2 * cos_i * nz
    horizon = np.array([0.780, 0.850, 0.920])
    sky = horizon + (SKY_ZENITH - horizon) * min(max(rz, 0.0), 1.0)
    for i in range(1, nx - 1):
        h = w[2, i] + d
        refr = WATER + (TERRAIN0 - WATER) / (1 + 0.5 * h)
        want = _bytes(R * sky + (1 - R) * refr)
        assert np.all(np.abs(img[2, i, :3].astype(int) - want) <= 1), i


def _plane_pixel(s, t, ex, view, h, absorb):
    """The Fresnel-mode colour of a plane water surface of slopes (s, t)
    under vertical exaggeration ex, seen along view, over a bed at zmin
    (terrain colour at t = 0) h below the surface: normal (-ex s, -ex t, 1)
    normalised, cos i = -I.n, reflected ray height I_z - 2 (I.n) n_z."""
    n = np.array([-ex * s, -ex * t, 1.0])
    n /= np.linalg.norm(n)
    I = np.asarray(view, float) / np.linalg.norm(view)
    idn = float(I @ n)
    R = _fresnel64(min(max(-idn, 0.0), 1.0))
    rz = I[2] - 2 * idn * n[2]
    horizon = np.array([0.780, 0.850, 0.920])
    sky = horizon + (SKY_ZENITH - horizon) * min(max(rz, 0.0), 1.0)
    refr = WATER + (TERRAIN0 - WATER) / (1 + absorb * h)
    return _bytes(R * sky + (1 - R) * refr), R


def test_tilted_plane_both_directions_grazing_view(oracle_mod):
    """A plane surface w = w_s + s x + t y (w_s = 0.7 m, dx != dy) seen at a
    grazing angle, where the reflection carries a quarter of the colour: the
    interior pixels follow the formula of the plane's normal in both
    directions, so the y-differences, both spacings and eta = w - w_s at
    every neighbour are all exercised."""
    nx, ny, dx, dy, s, t, ws, d = 12, 10, 0.1, 0.15, 0.4, -0.3, 0.7, 2.0
    x, y = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    w = ws + s * X + t * Y
    B = np.full((ny, nx), ws - d)
    view = (0.55, 0.7, -0.25)
    p = oracle_mod.render_params("fresnel", zmin=ws - d, zmax=ws + 1.0, absorb=0.3, exaggeration=1.5, view=view)
    img = oracle_mod.render(w, 0 * w, 0 * w, B, dx, dy, ws, p)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            want, R = _plane_pixel(s, t, 1.5, view, w[j, i] - B[j, i], 0.3)
            assert R > 0.2
            assert np.all(np.abs(img[j, i, :3].astype(int) - want) <= 1), (i, j)


def test_lake_shore_is_level(oracle_mod):
    """Still water at w_s = 0.7 m against dry land: a dry neighbour counts at
    the wet cell's own level, so the shore cells see a level surface and
    render as the open water does (the flat-lake formula seen obliquely)."""
    nx, ny, ws, d = 10, 8, 0.7, 1.5
    B = np.full((ny, nx), ws - d)
    B[:, 7:] = ws + 0.4                 # land east of column 6
    B[6:, :] = ws + 0.4                 # and north of row 5
    w = np.maximum(np.full((ny, nx), ws), B)
    view = (0.3, 0.5, -0.6)
    p = oracle_mod.render_params("fresnel", zmin=ws - d, zmax=ws + 1.0, absorb=0.3, view=view)
    img = oracle_mod.render(w, 0 * w, 0 * w, B, 0.2, 0.3, ws, p)
    want, _ = _plane_pixel(0.0, 0.0, 1.0, view, d, 0.3)
    wet = B < ws
    assert wet.sum() == 7 * 6
    assert np.all(np.abs(img[wet][:, :3].astype(int) - want) <= 1)


def test_colormap_range_of_the_value(oracle_mod):
    """The shown value is placed in [vmin, vmax] linearly: eta = 1 m on
    [-1, 3] m takes the colour at t = 1/2, eta = -1 m the colour at 0 and
    eta = 3 m the colour at 1."""
    B = np.full((3, 3), -4.0)
    for eta, tt in ((1.0, 0.5), (-1.0, 0.0), (3.0, 1.0), (0.0, 0.25)):
        w = np.full((3, 3), 0.5 + eta)
        img = oracle_mod.render(w, 0 * w, 0 * w, B, 1.0, 1.0, 0.5, oracle_mod.render_params("eta", vmin=-1.0, vmax=3.0))
        np.testing.assert_array_equal(img[1, 1, :3], _bytes(oracle_mod.colormap(0, tt)))


def test_hillshade_of_a_plane_in_both_directions(oracle_mod):
    """Land on a plane z = z0 + a x + b y under a sun with components along
    x, y and z: Lambert's shade 0.35 + 0.65 max(n.L, 0), n the plane's
    normal (-ex a, -ex b, 1) normalised, on the terrain colour of the cell,
    for the interior pixels (dx != dy)."""
    nx, ny, dx, dy, a, b, ex = 9, 7, 0.2, 0.3, 0.15, -0.1, 3.0
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)
    z = 1.0 + a * X + b * Y
    sun = (0.4, 0.6, 0.7)
    p = oracle_mod.render_params("eta", zmin=0.5, zmax=2.5, exaggeration=ex, sun=sun)
    img = oracle_mod.render(z, 0 * z, 0 * z, z, dx, dy, 0.0, p)
    n = np.array([-ex * a, -ex * b, 1.0])
    n /= np.linalg.norm(n)
    L = np.array(sun) / np.linalg.norm(sun)
    shade = 0.35 + 0.65 * max(float(n @ L), 0.0)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            terr = oracle_mod.colormap(2, (z[j, i] - 0.5) / 2.0).astype(np.float64)
            assert np.all(np.abs(img[j, i, :3].astype(int) - _bytes(terr * shade)) <= 1), (i, j)


def test_depth_equal_to_dry_h_is_land(oracle_mod):
    """A cell is land where w - Bbar <= dry_h: four neighbours of a lake cell
    hold exactly dry_h of water, their surface 0.25 m above the lake's, and
    still count as land, so they show the terrain and the lake cell between
    them sees a level surface."""
    dry_h, ws, d = 0.25, 0.0, 1.0
    B = np.full((3, 3), 0.5)
    w = B + dry_h                                   # depth dry_h exactly (all values exact in binary)
    B[1, 1], w[1, 1] = -d, ws
    view = (0.55, 0.7, -0.25)                        # grazing: the reflection weighs in
    p = oracle_mod.render_params("fresnel", dry_h=dry_h, zmin=-d, zmax=1.5, absorb=0.3, exaggeration=3.0,
                                 view=view)
    img = oracle_mod.render(w, 0 * w, 0 * w, B, 1.0, 1.0, ws, p)
    want, _ = _plane_pixel(0.0, 0.0, 3.0, view, d, 0.3)
    assert np.all(np.abs(img[1, 1, :3].astype(int) - want) <= 1)
    terr = oracle_mod.colormap(2, (0.5 + d) / 2.5).astype(np.float64)
    for (j, i) in ((0, 1), (2, 1), (1, 0), (1, 2)):
        # each land cell's bed is level towards its land neighbours and drops
        # towards the lake cell: not flat, so check only that it is land
        # coloured (no water term: its colour is a shade of the terrain's)
        px = img[j, i, :3].astype(np.float64) / 255.0
        ratio = px / terr
        assert np.allclose(ratio, ratio[0], atol=0.02)


@pytest.mark.parametrize("shape", [(1, 6), (6, 1), (1, 1)])
def test_one_cell_wide_strips_see_a_level_surface(oracle_mod, shape):
    """A strip one cell wide has no neighbour across it: the gradient there
    is taken as zero, so a lake strip renders as level water and a strip of
    flat land as flat land under the sun."""
    z = np.full(shape, 0.9)
    sun = (0.3, 0.4, 1.0)
    pl = oracle_mod.render_params("eta", zmin=0.5, zmax=1.5, sun=sun)
    land = oracle_mod.render(z, 0 * z, 0 * z, z, 0.5, 0.5, 0.0, pl)
    lz = 1.0 / np.linalg.norm(sun)
    want = _bytes(oracle_mod.colormap(2, 0.4).astype(np.float64) * (0.35 + 0.65 * lz))
    assert np.all(np.abs(land[..., :3].reshape(-1, 3).astype(int) - want) <= 1)
    ws, d = 0.2, 1.2
    w = np.full(shape, ws)
    B = np.full(shape, ws - d)
    view = (0.3, 0.5, -0.6)
    p = oracle_mod.render_params("fresnel", zmin=ws - d, zmax=ws + 1.0, absorb=0.3, view=view)
    img = oracle_mod.render(w, 0 * w, 0 * w, B, 0.5, 0.5, ws, p)
    want, _ = _plane_pixel(0.0, 0.0, 1.0, view, d, 0.3)
    assert np.all(np.abs(img[..., :3].reshape(-1, 3).astype(int) - want) <= 1)
