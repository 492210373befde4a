"""Pins of the tangent-linear oracle (oracle/celeris_tlm.cpp: the oracle's
own source compiled with forward-mode dual numbers), against things other
than itself:

* its values are the oracle's, bit for bit (the same arithmetic on the
  value parts);
* its tangents equal central differences of the plain oracle, in the bed
  and in the initial state, on a state away from the method's kinks,
  including where they run through the sine maker's and Manning's
  dependence on the depth;
* it is linear in the direction.
"""
import numpy as np

from tests.helpers import oracle_from, tangent_run, tilted_bed_scenario


def _oracle_eta(s, gauges, z=None, w0=None):
    import dataclasses
    o = oracle_from(dataclasses.replace(s, z=s.z if z is None else z))
    w, P, Q = s.initial_state()
    o.set_state(w if w0 is None else w0, P, Q)
    o.set_gauges(gauges, 1, s.steps)
    o.step(s.steps)
    return o.read_gauges(s.steps)


def _directions(X, Y, rng, n):
    out = []
    for _ in range(n):
        v = np.zeros_like(X)
        for _ in range(3):
            cx, cy = rng.uniform(2.0, 22.0), rng.uniform(2.0, 16.0)
            v += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(2.0, 8.0))
        out.append(v)
    return out


def test_tangent_oracle_values_are_the_oracles():
    s, gauges, X, _ = tilted_bed_scenario(model=0, K=1, sine=True)
    eta, _ = tangent_run(s, gauges, np.zeros_like(X), np.zeros_like(X))
    np.testing.assert_array_equal(eta, _oracle_eta(s, gauges))


def test_tangent_oracle_matches_central_differences():
    for model in (0, 1):
        s, gauges, X, Y = tilted_bed_scenario(model=model, K=1, friction=2, sine=True)
        rng = np.random.default_rng(5 + model)
        vz, vw = _directions(X, Y, rng, 2)
        vz *= 1e-2
        vw *= 1e-4
        _, deta = tangent_run(s, gauges, vz, vw)
        eps = 1e-5
        fd = (_oracle_eta(s, gauges, z=s.z + eps * vz, w0=s.w0 + eps * vw)
              - _oracle_eta(s, gauges, z=s.z - eps * vz, w0=s.w0 - eps * vw)) / (2 * eps)
        assert np.max(np.abs(deta - fd)) <= 1e-6 * np.max(np.abs(fd)), model


def test_tangent_oracle_is_linear_in_the_direction():
    s, gauges, X, Y = tilted_bed_scenario(model=0, K=1)
    rng = np.random.default_rng(8)
    a, b = _directions(X, Y, rng, 2)
    _, d1 = tangent_run(s, gauges, 1e-2 * a, 1e-4 * b)
    _, d2 = tangent_run(s, gauges, 1e-2 * b, 1e-4 * a)
    _, d3 = tangent_run(s, gauges, 1e-2 * (2 * a - 3 * b), 1e-4 * (2 * b - 3 * a))
    np.testing.assert_allclose(d3, 2 * d1 - 3 * d2, rtol=0, atol=1e-12 * np.max(np.abs(d3)))


def test_tangent_oracle_maker_and_manning_paths():
    """The same check where the tangent runs through the sine maker's
    dependence on the depth beside it (Eckart's k, the celerity, Eq. 25-29)
    and through Manning's depth-dependent coefficient (Eq. 32): bed
    directions on the two columns next to the maker, gauges near it, a
    2 cm maker and n = 0.05."""
    import dataclasses
    import math

    from paper_1611_05984_gb300 import scenarios as sc
    s, _, X, Y = tilted_bed_scenario(model=0, K=1, friction=2, sine=True, nsteps=12)
    s = dataclasses.replace(s, fcoef=0.05)
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.02, 3.0, 0.2, 0.3),))
    gauges = [(i, j) for i in (1, 3, 6) for j in (8, 18, 27)]
    for vz, vw in ((1e-2 * np.exp(-((X - 0.5) / 0.4) ** 2) * (1 + 0.3 * np.sin(2 * math.pi * Y / 9.0)), 0 * X),
                   (0 * X, 1e-4 * np.exp(-((X - 2.0) ** 2 + (Y - 9.0) ** 2) / 4.0))):
        _, deta = tangent_run(s, gauges, vz, vw)
        eps = 1e-5
        fd = (_oracle_eta(s, gauges, z=s.z + eps * vz, w0=s.w0 + eps * vw)
              - _oracle_eta(s, gauges, z=s.z - eps * vz, w0=s.w0 - eps * vw)) / (2 * eps)
        assert np.max(np.abs(fd)) > 0
        assert np.max(np.abs(deta - fd)) <= 1e-6 * np.max(np.abs(fd))
