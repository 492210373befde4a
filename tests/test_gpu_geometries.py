"""The paper's validation geometries (Sec. 4) on the CUDA path vs the oracle,
and run-up tracking (Sec. 4.1, 4.3) vs the oracle's.

Bars as in the other parity tests: relative L2 of eta = w - w_s, FP64 1e-10
and FP32 1e-4.  The run-up field is compared where both sides saw the cell
wet; which cells those are can differ only where a depth came within
rounding of the threshold at some step, so a few such cells are allowed and
counted.
"""
import math

import numpy as np
import pytest

from paper_1611_05984_gb300 import scenarios as sc
from tests.helpers import oracle_from, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


def _solver(s, prec):
    from paper_1611_05984_gb300 import celeris
    return celeris.from_scenario(s, dtype=torch.float64 if prec == "f64" else torch.float32)


def _np(t):
    return t.double().cpu().numpy()


def _lockstep(s, prec, nsteps, every, delta=None):
    o = oracle_from(s)
    g = _solver(s, prec)
    if delta is not None:
        o.runup_enable(delta)
        g.runup_enable(delta)
    done = 0
    while done < nsteps:
        n = min(every, nsteps - done)
        o.step(n)
        g.step(n)
        done += n
        e = rel_l2(_np(g.state()[0]) - s.ws, o.state()[0] - s.ws)
        assert e <= TOL[prec], f"eta rel-L2 {e:.3e} at step {done}"
    return o, g


def _compare_runup(o, g, prec):
    mo, mg = o.runup(), _np(g.runup())
    fo, fg = np.isfinite(mo), np.isfinite(mg)
    assert np.count_nonzero(fo != fg) <= max(2, fo.size // 2000)
    both = fo & fg
    assert np.count_nonzero(both) > 0
    assert rel_l2(mg[both], mo[both]) <= TOL[prec]
    return mo


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_whalin_shoal(prec):
    """Eq. 37 tank, 2000 x 65 (dx 1.75 cm, dy 9.4 cm), sine maker, 5 m sponge,
    400 steps of 1 ms."""
    s = sc.whalin()
    _lockstep(s, prec, 400, 100)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_planar_beach_runup(prec):
    """Breaking solitary wave (H/d = 0.28, f = 0.01) up a 1:19.85 beach
    through run-up and run-down, with run-up tracking at delta = s dx / 3."""
    s = sc.planar_beach_soliton(0.28, f=0.01)
    o, g = _lockstep(s, prec, s.steps, 250, delta=s.runup_delta)
    mo = _compare_runup(o, g, prec)
    bed = o.field("Bbar")
    assert np.any(np.isfinite(mo) & (bed > 0))     # the wave ran up the dry beach


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_conical_island_runup(prec):
    """Solitary wave (H/d = 0.18) onto the conical island, 301 x 301 cells
    (dx 10 cm), 1400 steps of 5 ms: up to run-up on the island's front face."""
    s = sc.conical_island(0.18, n=301)
    o, g = _lockstep(s, prec, 1400, 350, delta=s.runup_delta)
    mo = _compare_runup(o, g, prec)
    bed = o.field("Bbar")
    assert np.any(np.isfinite(mo) & (bed > 0))


def test_runup_tracking_starts_from_state_and_disables():
    s = sc.planar_beach_soliton(0.05)
    g = _solver(s, "f32")
    g.runup_enable(s.runup_delta)
    w = _np(g.state()[0])
    bed = _np(g.field("Bbar"))
    m = _np(g.runup())
    wet = w - bed > s.runup_delta
    np.testing.assert_array_equal(np.isfinite(m), wet)
    np.testing.assert_array_equal(m[wet], w[wet])
    g.step(5)
    tracked = g.last_launch_count()
    g.runup_disable()
    g2 = _solver(s, "f32")
    g2.step(5)
    assert tracked == g2.last_launch_count() + 5        # one run-up launch per step
    g.set_state(*g2.state())
    g.step(5)
    g2.set_state(*g2.state())   # both restart their history past the first call (which builds the sponge table)
    g2.step(5)
    assert g.last_launch_count() == g2.last_launch_count()   # none once disabled


def test_planar_beach_nonbreaking_runup_law():
    """A non-breaking solitary wave (H/d = 0.005, dx/d = 0.0625) on the
    1:19.85 beach: the maximum run-up is within 15 % of the run-up law
    R/d = 2.831 sqrt(cot beta) (H/d)^(5/4) (Synolakis 1987), which the
    paper's Fig. 6 compares against."""
    from paper_1611_05984_gb300 import validation
    H = 0.005
    s = sc.planar_beach_soliton(H)
    g = _solver(s, "f32")
    g.runup_enable(s.runup_delta)
    g.step(s.steps)
    assert g.check_finite()
    R = validation.vertical_runup(_np(g.runup()), _np(g.field("Bbar")))
    law = 2.831 * math.sqrt(19.85) * H ** 1.25
    assert abs(R / law - 1.0) <= 0.15
