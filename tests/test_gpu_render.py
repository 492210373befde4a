"""Headless renderer (cel_render) vs the render oracle, byte for byte.

Both sides compute in single precision one rounded operation at a time, so
every byte must agree.  The state is a beach crop after its sine waves have
run up the shore (wet and dry cells, a moving shoreline), rendered in every
mode; the oracle gets the same w, P, Q and cell bed that the solver holds.
"""
import numpy as np
import pytest

from paper_1611_05984_gb300 import scenarios as sc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _state(prec, nx=200, ny=150, steps=400):
    from paper_1611_05984_gb300 import celeris
    s = sc.beach(nx=nx, ny=ny, sponge=20)
    g = celeris.from_scenario(s, dtype=torch.float64 if prec == "f64" else torch.float32)
    g.step(steps)
    return s, g


def _oracle_image(oracle_mod, s, g, kw):
    w, P, Q = (t.double().cpu().numpy() for t in g.state())
    B = g.field("Bbar").double().cpu().numpy()
    return oracle_mod.render(w, P, Q, B, s.dx, s.dy, s.ws, oracle_mod.render_params(**kw))


CASES = [
    dict(mode="eta", vmin=-0.4, vmax=0.4, zmin=-10.0, zmax=3.0),
    dict(mode="u", vmin=-1.0, vmax=1.0, zmin=-10.0, zmax=3.0, h_min=0.05),
    dict(mode="v", vmin=-0.3, vmax=0.3, zmin=-10.0, zmax=3.0),
    dict(mode="speed", vmin=0.0, vmax=1.5, zmin=-10.0, zmax=3.0, grid=25.0),
    dict(mode="fresnel", zmin=-10.0, zmax=3.0, exaggeration=20.0, view=(0.5, 0.3, -0.8), sun=(0.4, 0.2, 1.0),
         absorb=0.3),
    dict(mode="fresnel", zmin=-10.0, zmax=3.0, exaggeration=1.0, view=(0.0, 0.0, -1.0), grid=10.0,
         dry_h=0.05),
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_render_matches_oracle_bytes(oracle_mod, prec):
    from paper_1611_05984_gb300 import celeris
    s, g = _state(prec)
    for kw in CASES:
        img = g.render(celeris.render_params(**kw)).cpu().numpy()
        ref = _oracle_image(oracle_mod, s, g, kw)
        bad = np.count_nonzero(np.any(img != ref, axis=-1))
        assert bad == 0, f"{kw['mode']}: {bad} pixels differ"
    # the image shows both water and land
    B = g.field("Bbar").double().cpu().numpy()
    assert np.any(B > 0) and np.any(B < 0)


def test_render_ragged_tiny_grid(oracle_mod):
    """A 37 x 5 grid (partial tiles, one-sided edge gradients) and a 1-row
    halo clamp in every direction."""
    from paper_1611_05984_gb300 import celeris
    s, g = _state("f32", nx=37, ny=5, steps=60)
    for kw in CASES:
        img = g.render(celeris.render_params(**kw)).cpu().numpy()
        np.testing.assert_array_equal(img, _oracle_image(oracle_mod, s, g, kw))


def test_render_rejects_bad_parameters():
    from paper_1611_05984_gb300 import celeris
    s, g = _state("f32", nx=40, ny=40, steps=1)
    for kw in (dict(vmin=1.0, vmax=1.0), dict(mode=7), dict(view=(0.0, 0.0, 0.0)), dict(h_min=0.0),
               dict(grid=-1.0), dict(zmin=2.0, zmax=1.0)):
        with pytest.raises(celeris.CelerisError):
            g.render(celeris.render_params(**kw))
