"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form,
an invariant, a textbook routine, a special case or a convergence order.

  Part of the oracle                      Pin (test below)
  --------------------------------------  --------------------------------------
  Thomas solver (Eq. 21-23 solves)        dense LAPACK solve        test_thomas_*
  minmod (KP07 step 1)                    hand cases                test_minmod_*
  Eckart k (Eq. 29)                       Newton on w^2 = gk tanh kd test_eckart_*
  sponge gamma (Eq. 30)                   end values, monotone      test_sponge_*
  central-upwind flux (KP07 step 3)       consistency, upwinding,   test_central_*
                                          mirror symmetry
  reconstruction + flux + bed slope       lake at rest              test_lake_*
  flux form, walls, AB3 / AM4             mass conservation         test_mass_*
  NLSW path, dry front                    Ritter closed form        test_ritter_*
  dispersion terms, tridiagonal, F*, G*   linear dispersion relation test_dispersion_*
  depth-gradient terms of Eq. 10-11       linear shoaling           test_linear_shoaling_*
  depth-gradient terms of F*, G* and      isotropy over a round     test_isotropy_*
  the cross terms of Eq. 10-11            shoal (axes vs diagonals)
  corner ghosts (Reading A-B5)            embedding beside a wall;  test_corner_ghost*
                                          plane wave of two makers
  NLSW reduction at d = 0 (Sec. 2.1)      the two models agree       test_boussinesq_reduces_*
  ghosts, x/y treatment                   mirror / transpose symmetry test_symmetry_*
  positivity fix, dry clamp               symmetry with wet-dry fronts test_symmetry_mirror_x_wet_dry
  positivity fix on the y-faces           the wet-dry basin along y  test_symmetry_transpose_wet_dry
  maker beside dry land (d = 0)           sends nothing, stays dry  test_sine_maker_beside_dry_land
  dry clamp and dry discharges (A-D1)     w >= bed, P = Q = 0 dry,  test_dry_land_*
                                          mass less the clamp's
                                          addition conserved
  gauges                                  eta about w_s, ring       test_gauges_*, test_gauge_ring
  sponge relaxation to w_s                still water stays still   test_lake_at_rest_with_sponges_*
  sponge on dry land                      land stays on its bed     test_sponge_leaves_dry_land_*
  sponge distances and widths in metres   one step of a raised lake test_sponge_profile_in_metres
  east and north makers                   mirrored runs             test_symmetry_mirror_sine_makers
  soliton (Eq. 33-36) + propagation       crest speed c_s (Eq. 36), test_soliton_*
                                          the profile's volume
  soliton direction                       transposed runs           test_symmetry_transpose_solitons
  soliton heading, width at d != 1        M parallel to grad eta,   test_solitary_wave_heading_*
                                          volume at d = 0.5 m
  parameter checks                        refusals                  test_oracle_refuses_*
  sine maker (Eq. 25-29)                  progressive wave P = c eta test_sine_maker_*
  sine maker on the y-sides               transposed runs           test_symmetry_transpose_sine_*
  friction (Eq. 31-32) + start-up + AB3   ODE closed form, orders;  test_friction_*
                                          oblique uniform flow
  AM4 weights of w, start-up F*, G*       1-D mode with corrector;  test_dispersion_relation_1d_with_*
  increments (Sec. 2.3, Eq. 18)           mode started from its     test_standing_mode_started_*
                                          discharges
  AB3 stability (Sec. 2.3)                real-axis bound -6/11     test_stability_*
"""
import math

import numpy as np
import pytest

from paper_1611_05984_gb300 import scenarios as sc
from tests.helpers import oracle_from

G = 9.81
B = 1.0 / 15.0


# --------------------------------------------------------------- pieces

def test_thomas_vs_dense(oracle_mod):
    rng = np.random.default_rng(11)
    for n in list(range(1, 33)) + [97, 256]:
        a = rng.uniform(-1, 1, n)
        c = rng.uniform(-1, 1, n)
        a[0] = 0.0
        c[-1] = 0.0
        b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 2.0, n)
        b *= rng.choice([-1.0, 1.0], n)
        r = rng.standard_normal(n)
        M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        x = oracle_mod.thomas(a, b, c, r)
        ref = np.linalg.solve(M, r)
        assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_minmod_cases(oracle_mod):
    mm = oracle_mod.minmod
    assert mm(1.3, 0.0, 1.0, 2.0) == pytest.approx(1.0)        # linear: central
    assert mm(1.3, 0.0, 1.0, 1.1) == pytest.approx(0.13)       # theta * forward
    assert mm(2.0, 0.0, 0.1, 5.0) == pytest.approx(0.2)        # theta * backward
    assert mm(1.3, 0.0, 1.0, 0.5) == 0.0                       # extremum
    assert mm(1.3, 2.0, 1.0, 0.0) == pytest.approx(-1.0)       # decreasing
    assert mm(1.0, 0.0, 1.0, 3.0) == pytest.approx(1.0)        # theta=1: minmod(fwd,bwd)


def _airy_k(omega, d):
    k = omega / math.sqrt(G * d)
    for _ in range(100):
        f = G * k * math.tanh(k * d) - omega ** 2
        fp = G * math.tanh(k * d) + G * k * d / math.cosh(k * d) ** 2
        k -= f / fp
    return k


def test_eckart_vs_exact_dispersion(oracle_mod):
    d = 1.0
    for kd in np.geomspace(0.05, 10.0, 40):
        k = kd / d
        omega = math.sqrt(G * k * math.tanh(kd))
        ke = oracle_mod.eckart_k(omega, d)
        assert abs(ke / _airy_k(omega, d) - 1.0) < 0.06
    # limits: deep water k = w^2/g; shallow k -> w/sqrt(gd)
    om = 10.0
    assert oracle_mod.eckart_k(om, 50.0) == pytest.approx(om * om / G, rel=1e-12)
    om = 0.01
    assert oracle_mod.eckart_k(om, 1.0) == pytest.approx(om / math.sqrt(G), rel=1e-4)


def test_sponge_gamma(oracle_mod):
    g = oracle_mod.sponge_gamma
    L = 20.0
    assert g(0.0, L) == pytest.approx(0.0, abs=1e-15)
    assert g(L, L) == 1.0
    assert g(5 * L, L) == 1.0
    assert g(0.5 * L, L) == pytest.approx(0.5)
    v = [g(D, L) for D in np.linspace(0, L, 101)]
    assert all(b >= a for a, b in zip(v, v[1:]))


def test_central_upwind_consistency(oracle_mod):
    cu = oracle_mod.central_upwind
    eps = 5e-12
    # identical states: flux equals the physical flux F(U) (Eq. 1)
    h, u, v, Bf = 2.0, 0.7, -0.3, -1.5
    w = Bf + h
    H = cu(G, eps, w, h * u, h * v, w, h * u, h * v, Bf)
    assert H == pytest.approx([h * u, h * u * u + 0.5 * G * h * h, h * u * v], rel=1e-13)
    # lake at rest: hydrostatic momentum flux only
    H = cu(G, eps, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -3.0)
    assert H == pytest.approx([0.0, 0.5 * G * 9.0, 0.0], abs=1e-13)
    # supercritical to the right: pure upwinding, H = F(U_left), the
    # tangential velocity carried from the left as well
    hL, uL, vL, hR, uR, vR = 0.5, 10.0, 1.5, 0.4, 9.0, -2.0
    H = cu(G, eps, hL, hL * uL, hL * vL, hR, hR * uR, hR * vR, 0.0)
    assert H == pytest.approx([hL * uL, hL * uL * uL + 0.5 * G * hL * hL, hL * uL * vL], rel=1e-12)
    # and supercritical to the left: H = F(U_right)
    H = cu(G, eps, hR, -hR * uR, hR * vR, hL, -hL * uL, hL * vL, 0.0)
    assert H == pytest.approx([-hL * uL, hL * uL * uL + 0.5 * G * hL * hL, -hL * uL * vL], rel=1e-12)
    # both sides dry
    assert list(cu(G, eps, 1.0, 0.3, 0.1, 1.0, -0.2, 0.0, 1.0)) == [0.0, 0.0, 0.0]


def test_central_upwind_mirror_symmetry(oracle_mod):
    """KP07 step 3 is unchanged by the reflection x -> -x: the face's sides
    trade places, the normal discharges change sign, the one-sided speeds
    a+ and a- trade places with a sign, so the flux through the reflected
    face is (-H0, H1, -H2).  A speed taken from the wrong side, or a sign
    slip in one of the two fluxes, breaks it.  Seeded random states, some
    sides dry."""
    cu = oracle_mod.central_upwind
    rng = np.random.default_rng(1611)
    for _ in range(400):
        Bf = rng.uniform(-2.0, 0.5)
        hL, hR = (0.0 if rng.random() < 0.15 else rng.uniform(0.0, 3.0) for _ in range(2))
        nL, tL, nR, tR = rng.uniform(-6.0, 6.0, 4)
        wL, wR = Bf + hL, Bf + hR
        H = cu(G, 5e-12, wL, nL, tL, wR, nR, tR, Bf)
        Hm = cu(G, 5e-12, wR, -nR, tR, wL, -nL, tL, Bf)
        scale = max(1.0, max(abs(v) for v in H))
        assert Hm[0] == pytest.approx(-H[0], rel=1e-13, abs=1e-13 * scale)
        assert Hm[1] == pytest.approx(H[1], rel=1e-13, abs=1e-13 * scale)
        assert Hm[2] == pytest.approx(-H[2], rel=1e-13, abs=1e-13 * scale)


# -------------------------------------------------------------- invariants

def test_lake_at_rest_submerged(oracle_mod):
    """KP07 with corner bed values is exactly well-balanced when submerged."""
    nx, ny = 64, 48
    z = sc.random_bed(nx, ny, 5, -9.0, -1.0, smooth=2)
    dmax = 9.0
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.1 / math.sqrt(G * dmax), K=1,
                          friction=2, fcoef=0.015)
    o.set_state(np.zeros_like(z), np.zeros_like(z), np.zeros_like(z))
    o.step(1000)
    w, P, Q = o.state()
    bound = 1e-12 * math.sqrt(G * dmax) * dmax
    assert np.max(np.abs(P)) <= bound and np.max(np.abs(Q)) <= bound
    assert np.max(np.abs(w)) <= 1e-13


def test_lake_at_rest_with_sponges_off_zero_level(oracle_mod):
    """Still water at a level w_s = 0.3 m (Sec. 2.1) over a submerged bed,
    sponges on all four sides (Eq. 30): the sponge relaxes towards w_s, so
    the lake stays exactly at rest."""
    nx, ny, ws = 48, 40, 0.3
    z = sc.random_bed(nx, ny, 7, -6.0, -0.5, smooth=2) + ws
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.1 / math.sqrt(G * 6.0), K=1, ws=ws)
    for side in (oracle_mod.W, oracle_mod.E, oracle_mod.S, oracle_mod.N):
        o.set_boundary(side, oracle_mod.SPONGE, 6)
    o.set_state(np.full_like(z, ws), np.zeros_like(z), np.zeros_like(z))
    o.step(300)
    w, P, Q = o.state()
    assert np.max(np.abs(w - ws)) <= 1e-13
    assert np.max(np.abs(P)) <= 1e-12 and np.max(np.abs(Q)) <= 1e-12


def test_sponge_leaves_dry_land_at_its_bed(oracle_mod):
    """Eq. 30 damps the free surface towards the still-water level w_s; land
    above w_s inside the layer holds no water, so its surface stays on its
    bed (a relaxation of w there would pull it 0.2 m below the bed).  A lake
    against a cliff to land 0.2 m above w_s, the land inside an east sponge."""
    nx, ny = 60, 8
    z = np.full((ny, nx), -0.5)
    z[:, 50:] = 0.2
    o = oracle_mod.Oracle(z, 0.1, 0.1, 0.01, K=1)
    o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, 15)
    o.set_state(0 * z, 0 * z, 0 * z)
    o.step(50)
    w, P, Q = o.state()
    Bbar = o.field("Bbar")
    assert np.all(w >= Bbar)
    np.testing.assert_array_equal(w[:, 51:], Bbar[:, 51:])
    assert np.all(P[:, 51:] == 0.0) and np.all(Q[:, 51:] == 0.0)


@pytest.mark.parametrize("K", [0, 2])
def test_mass_soliton_channel(oracle_mod, K):
    s = sc.soliton_channel(K=K)
    o = oracle_from(s)
    m0 = o.mass()
    o.step(1000)
    assert o.clamp_mass() == 0.0
    assert abs(o.mass() - m0) <= 1e-13 * abs(m0)


def test_mass_2d_closed_basin(oracle_mod):
    nx, ny = 64, 48
    z = sc.random_bed(nx, ny, 7, -3.0, -1.0, smooth=3)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    eta = 0.2 * np.exp(-((X - 20) ** 2 + (Y - 25) ** 2) / 30.0)
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.1 / math.sqrt(G * 3.0), K=1,
                          friction=2, fcoef=0.02)
    o.set_state(eta, 0 * z, 0 * z)
    m0 = o.mass()
    o.step(1000)
    assert o.clamp_mass() == 0.0
    assert abs(o.mass() - m0) <= 1e-13 * abs(m0)


# ------------------------------------------------------------ closed forms

def _ritter_l1(oracle_mod, dx, T=1.5):
    L0, L1 = -8.0, 12.0
    nx, ny = int(round((L1 - L0) / dx)), 2
    x = L0 + (np.arange(nx) + 0.5) * dx
    z = np.zeros((ny, nx))
    dt = 0.1 * dx / math.sqrt(G)      # front moves at 2 sqrt(g h0)
    o = oracle_mod.Oracle(z, dx, dx, dt, model=oracle_mod.NLSW)
    o.set_state(np.tile(np.where(x < 0, 1.0, 0.0), (ny, 1)), 0 * z, 0 * z)
    n = int(round(T / dt))
    o.step(n)
    t = n * dt
    w, _, _ = o.state()
    c0 = math.sqrt(G)
    h_ex = np.where(x < -c0 * t, 1.0,
                    np.where(x > 2 * c0 * t, 0.0, (2 * c0 - x / t) ** 2 / (9 * G)))
    m = (x > -c0 * t - 1.0) & (x < 2 * c0 * t + 1.0)
    assert np.array_equal(w[0], w[1])
    return float(np.sum(np.abs(w[0] - h_ex)[m]) / np.sum(h_ex[m]))


def test_ritter_dam_break(oracle_mod):
    e1 = _ritter_l1(oracle_mod, 0.02)
    e2 = _ritter_l1(oracle_mod, 0.01)
    assert e2 <= 0.02 and e1 <= 0.02
    assert e2 < 0.75 * e1


def _omega(k, d):
    return k * math.sqrt(G * d * (1 + B * (k * d) ** 2) / (1 + (B + 1 / 3) * (k * d) ** 2))


def _standing_period_error(oracle_mod, kd, cpl, twod=False, periods=3, K=None):
    """Standing mode eta = a cos(kx x)[cos(ky y)] in a walled basin; period
    from the zero crossings of eta at the corner cell vs the linear
    dispersion relation of Eq. 2 / 7 / 10 (flat bed).  K defaults to 1 for
    the oblique mode and 0 for the 1-D one."""
    d = 1.0
    k = kd / d
    if twod:
        kx = ky = k / math.sqrt(2)
        nx = ny = cpl
    else:
        kx, ky, nx, ny = k, 0.0, cpl, 2
    dx = 2 * math.pi / kx / cpl
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    eta = 1e-4 * d * np.cos(kx * X) * (np.cos(ky * Y) if twod else 1.0)
    z = np.full((ny, nx), -d)
    dt = 0.2 * dx / math.sqrt(G * d)
    o = oracle_mod.Oracle(z, dx, dx, dt, K=(1 if twod else 0) if K is None else K)
    o.set_state(eta, 0 * z, 0 * z)
    T = 2 * math.pi / _omega(k, d)
    n = int(periods * T / dt) + 2
    sig = np.empty(n)
    for s in range(n):
        o.step(1)
        sig[s] = o.state()[0][0, 0]
    t = (np.arange(n) + 1) * dt
    zc = [t[s] - sig[s] * dt / (sig[s + 1] - sig[s])
          for s in range(n - 1) if sig[s] * sig[s + 1] < 0]
    return abs(2 * np.mean(np.diff(zc)) / T - 1)


@pytest.mark.parametrize("kd", [0.5, 1.0, 2.0, 3.0])
def test_dispersion_relation_1d(oracle_mod, kd):
    e64 = _standing_period_error(oracle_mod, kd, 64)
    e128 = _standing_period_error(oracle_mod, kd, 128)
    assert e64 <= 5e-3
    assert e128 <= e64 / 3.0          # second order in space


@pytest.mark.parametrize("kd", [1.0, 2.0])
def test_dispersion_relation_1d_with_corrector(oracle_mod, kd):
    """The same 1-D mode with one AM4 corrector iteration (Eq. 18-20): the
    corrector's weights of w and of U must keep the period, to second order
    in space."""
    e64 = _standing_period_error(oracle_mod, kd, 64, K=1)
    e128 = _standing_period_error(oracle_mod, kd, 128, K=1)
    assert e64 <= 5e-3
    assert e128 <= e64 / 3.0


@pytest.mark.parametrize("kd", [1.0, 2.0])
def test_dispersion_relation_2d_oblique(oracle_mod, kd):
    """An oblique mode needs the mixed terms of Eq. 10-13 (F*, G*, eta_xyy)."""
    e32 = _standing_period_error(oracle_mod, kd, 32, twod=True)
    e64 = _standing_period_error(oracle_mod, kd, 64, twod=True)
    assert e64 <= 5e-3
    assert e64 <= e32 / 3.0


def _moving_standing_mode(oracle_mod, kd, cpl, periods=2.0):
    """The oblique standing mode of the test above, started a quarter period
    later: eta = 0 and the discharges (P, Q) = grad phi that continuity
    (eta_t + P_x + Q_y = 0) gives for eta = a cos(kx x) cos(ky y) cos(omega t),
    omega from the dispersion relation of Eq. 2 / 7 / 10.  Then
    eta = -a cos(kx x) cos(ky y) sin(omega t).  Returns the fitted sine and
    cosine amplitudes of eta at the corner cell, over a (1 and 0 exactly)."""
    d = 1.0
    k = kd / d
    kx = ky = k / math.sqrt(2)
    dx = 2 * math.pi / kx / cpl
    X, Y = np.meshgrid((np.arange(cpl) + 0.5) * dx, (np.arange(cpl) + 0.5) * dx)
    a, om = 1e-4 * d, _omega(k, d)
    P = a * om * kx / k ** 2 * np.sin(kx * X) * np.cos(ky * Y)
    Q = a * om * ky / k ** 2 * np.cos(kx * X) * np.sin(ky * Y)
    z = np.full((cpl, cpl), -d)
    dt = 0.2 * dx / math.sqrt(G * d)
    o = oracle_mod.Oracle(z, dx, dx, dt, K=1)
    o.set_state(0 * z, P, Q)
    n = int(periods * 2 * math.pi / om / dt) + 2
    sig = np.empty(n)
    for s in range(n):
        o.step(1)
        sig[s] = o.state()[0][0, 0]
    t = (np.arange(n) + 1) * dt
    corner = a * math.cos(kx * 0.5 * dx) * math.cos(ky * 0.5 * dx)
    A = np.stack([np.sin(om * t), np.cos(om * t)], 1)
    cs, cc = np.linalg.lstsq(A, sig, rcond=None)[0]
    return -cs / corner, cc / corner


@pytest.mark.parametrize("kd", [1.0, 2.0])
def test_standing_mode_started_from_its_discharges(oracle_mod, kd):
    """With discharges at t = 0 the mixed terms F*, G* (Eq. 12-13) are not
    zero at the start, so the start-up steps' F* and G* increments (Sec. 2.3:
    none on the first step, F*^1 - F*^0 on the second) and the AM4 weights
    of w (Eq. 18) all shape the first periods: eta must come back with the
    amplitude and phase of the linear mode, converging in space."""
    s32, c32 = _moving_standing_mode(oracle_mod, kd, 32)
    s64, c64 = _moving_standing_mode(oracle_mod, kd, 64)
    assert abs(s64 - 1) <= 5e-3
    assert abs(c64) <= 1e-2
    assert abs(s64 - 1) <= abs(s32 - 1) / 3.0


def test_soliton_speed(oracle_mod):
    """Eq. 33-36 on a long flat channel: crest speed c_s = sqrt(g(H+d))."""
    H, d, dx, ny = 0.1, 1.0, 0.05, 2
    nx = int(130.0 / dx)
    z = np.full((ny, nx), -d)
    dt = 0.2 * dx / math.sqrt(G * d)
    o = oracle_mod.Oracle(z, dx, dx, dt)
    o.set_state(0 * z, 0 * z, 0 * z)
    o.add_solitary(H, 0.0, 15.0, ny * dx / 2)
    x = (np.arange(nx) + 0.5) * dx

    def crest():
        w = o.state()[0][0]
        i = int(np.argmax(w))
        y0, y1, y2 = w[i - 1], w[i], w[i + 1]
        return x[i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * dx, y1

    n1, n2 = int(5.0 / dt), int(30.0 / dt)
    o.step(n1)
    xa, ha = crest()
    o.step(n2 - n1)
    xb, hb = crest()
    c = (xb - xa) / ((n2 - n1) * dt)
    assert abs(c / math.sqrt(G * (H + d)) - 1) <= 0.03
    assert hb >= 0.95 * H
    # the volume of Eq. 33's sech^2 profile over the channel, per unit crest
    # length: the integral of H sech^2(k (x - x0)) from 0 to L (the flux form
    # keeps it while the wave travels)
    k = math.sqrt(3 * H / (4 * d ** 3))
    vol = o.state()[0][0].sum() * dx
    exact = H / k * (math.tanh(k * (nx * dx - 15.0)) + math.tanh(k * 15.0))
    assert vol == pytest.approx(exact, rel=1e-4)


def test_solitary_wave_heading_and_depth(oracle_mod):
    """Eq. 33-36 describe a wave travelling along its heading n = (cos
    theta, sin theta): its discharge c eta n is normal to its crest, so M
    is parallel to grad eta wherever the wave stands out (a heading of 30
    degrees, where neither component vanishes); and its width follows the
    still-water depth d at the crest: at d = 0.5 m the channel holds the
    volume of H sech^2(k (x - x0)), k = sqrt(3 H / (4 d^3))."""
    n, dx, d, H = 120, 0.1, 0.5, 0.025
    z = np.full((n, n), -d)
    o = oracle_mod.Oracle(z, dx, dx, 0.01, K=1)
    o.set_state(0 * z, 0 * z, 0 * z)
    o.add_solitary(H, math.radians(30), 6.0, 6.0)
    w, P, Q = o.state()
    ex = (w[1:-1, 2:] - w[1:-1, :-2]) / (2 * dx)
    ey = (w[2:, 1:-1] - w[:-2, 1:-1]) / (2 * dx)
    Pi, Qi = P[1:-1, 1:-1], Q[1:-1, 1:-1]
    m = w[1:-1, 1:-1] > 0.2 * H
    cross = np.abs(Pi * ey - Qi * ex)[m]
    scale = (np.hypot(Pi, Qi) * np.hypot(ex, ey))[m]
    assert m.sum() > 1000 and np.max(cross / np.maximum(scale, 1e-300)) <= 1e-2
    assert np.all(Qi[m] > 0) and np.all(Pi[m] > 0)
    # the width at d = 0.5 m: a straight crest across a channel
    nx, ny = 400, 4
    zc = np.full((ny, nx), -d)
    oc = oracle_mod.Oracle(zc, dx, dx, 0.01)
    oc.set_state(0 * zc, 0 * zc, 0 * zc)
    oc.add_solitary(H, 0.0, 15.0, ny * dx / 2)
    k = math.sqrt(3 * H / (4 * d ** 3))
    vol = oc.state()[0][0].sum() * dx
    assert vol == pytest.approx(H / k * (math.tanh(k * (nx * dx - 15.0)) + math.tanh(k * 15.0)), rel=1e-4)


def test_oracle_refuses_invalid_parameters(oracle_mod):
    """orc_create refuses a grid of fewer than 2 x 2 cells and spacings,
    a step or an epsilon that are not positive, and a negative K."""
    z = np.full((4, 4), -1.0)
    good = dict(dx=0.5, dy=0.5, dt=0.01)
    oracle_mod.Oracle(z, good["dx"], good["dy"], good["dt"])
    for dx, dy, dt, kw in ((0.0, 0.5, 0.01, {}), (0.5, 0.0, 0.01, {}), (0.5, 0.5, 0.0, {}),
                           (0.5, 0.5, 0.01, {"eps": 0.0}), (0.5, 0.5, 0.01, {"K": -1})):
        with pytest.raises(ValueError):
            oracle_mod.Oracle(z, dx, dy, dt, **kw)
    with pytest.raises(ValueError):
        oracle_mod.Oracle(np.full((1, 4), -1.0), 0.5, 0.5, 0.01)


def _uniform_friction_error(oracle_mod, dt, f=0.5, P0=0.5, h=1.0, T=2.0, kind=1):
    nx, ny, dx = 400, 2, 0.1
    z = np.full((ny, nx), -h)
    o = oracle_mod.Oracle(z, dx, dx, dt, model=oracle_mod.NLSW, friction=kind, fcoef=f)
    o.set_state(0 * z, P0 + 0 * z, 0 * z)
    n = int(round(T / dt))
    o.step(n)
    return o.state()[1][0, nx // 2], n * dt


def test_friction_quadratic_order(oracle_mod):
    """Eq. 31 with constant f on a uniform flow: P' = -f P|P|/h^2, exactly
    P(t) = P0/(1 + f P0 t/h^2).  The two forward-Euler start-up steps
    (Sec. 2.3) give the O(dt^2) error -2 a^2 P0^3 dt^2/(1 + a P0 T)^2,
    a = f/h^2; what remains is the AB3 error, O(dt^3)."""
    f, P0, h = 0.5, 0.5, 1.0
    a = f / h ** 2
    res = []
    for dt in (0.008, 0.004, 0.002):
        P, T = _uniform_friction_error(oracle_mod, dt, f=f, P0=P0, h=h)
        err = P - P0 / (1 + a * P0 * T)
        startup = -2 * a * a * P0 ** 3 * dt * dt / (1 + a * P0 * T) ** 2
        assert err == pytest.approx(startup, rel=0.05)
        res.append(abs(err - startup))
    assert math.log2(res[0] / res[1]) >= 2.7
    assert math.log2(res[1] / res[2]) >= 2.7


def test_friction_manning_ode(oracle_mod):
    """Eq. 32: f = g n^2 / h^(1/3); compare with a quadrature of the ODE."""
    from scipy.integrate import solve_ivp
    n_m, P0, h, T = 0.03, 0.8, 0.5, 2.0
    fm = G * n_m ** 2 / h ** (1 / 3)
    sol = solve_ivp(lambda t, p: -fm * p * np.abs(p) / h ** 2, (0, T), [P0],
                    rtol=1e-12, atol=1e-14)
    ref = sol.y[0, -1]
    P, _ = _uniform_friction_error(oracle_mod, 0.002, f=n_m, P0=P0, h=h, T=T, kind=2)
    assert P == pytest.approx(ref, rel=1e-5)


def test_friction_quadratic_oblique_flow(oracle_mod):
    """Eq. 31 acts on the discharge vector M = (P, Q) through its length:
    M' = -f M |M| / h^2 on a uniform flow, so the direction of M stays put
    and |M| follows the 1-D solution |M0| / (1 + f |M0| t / h^2), less the
    forward-Euler start-up term of the test above (h = 0.6 m, so the
    1/h^2 of Eq. 31 shows in both components)."""
    f, h, T, dt = 0.5, 0.6, 2.0, 0.004
    P0, Q0 = 0.4, 0.3
    M0, a = math.hypot(P0, Q0), f / h ** 2
    nx, ny, dx = 200, 200, 0.1
    z = np.full((ny, nx), -h)
    o = oracle_mod.Oracle(z, dx, dx, dt, model=oracle_mod.NLSW, friction=1, fcoef=f)
    o.set_state(0 * z, P0 + 0 * z, Q0 + 0 * z)
    o.step(int(round(T / dt)))
    _, P, Q = o.state()
    p, q = P[ny // 2, nx // 2], Q[ny // 2, nx // 2]
    assert q / p == pytest.approx(Q0 / P0, rel=1e-12)
    startup = -2 * a * a * M0 ** 3 * dt * dt / (1 + a * M0 * T) ** 2
    assert math.hypot(p, q) - M0 / (1 + a * M0 * T) == pytest.approx(startup, rel=0.05)


# ------------------------------------------------------------ sine maker

def _sine_channel(oracle_mod, courant, d=1.0, a=0.005, T=4.0, dx=0.1, ny=2):
    """West sine maker, east sponge two wavelengths wide, Boussinesq, K = 1,
    from rest; after 5 periods, the amplitude and phase of eta and P at the
    frequency of the maker over 2 periods, at 0.5 and 1 wavelength from it."""
    w0 = 2 * math.pi / T
    L = 2 * math.pi / oracle_mod.eckart_k(w0, d, G)
    nx, sponge = int(round(6 * L / dx)), int(round(2 * L / dx))
    z = np.full((ny, nx), -d)
    dt = courant * dx / math.sqrt(G * d)
    o = oracle_mod.Oracle(z, dx, dx, dt, K=1)
    o.set_boundary(oracle_mod.W, oracle_mod.SINE, 0, ((a, T, 0.0, 0.0),))
    o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, sponge)
    o.set_state(0 * z, 0 * z, 0 * z)
    n_total, n_fit = int(round(7 * T / dt)), int(round(2 * T / dt))
    o.step(n_total - n_fit)
    gi = [int(round(f * L / dx)) for f in (0.5, 1.0)]
    t, eta, P = [], [], []
    for n in range(n_fit):
        o.step(1)
        w, p, _ = o.state()
        t.append((n_total - n_fit + n + 1) * dt)
        eta.append(w[0, gi])
        P.append(p[0, gi])
    t = np.array(t)
    A = np.stack([np.cos(w0 * t), np.sin(w0 * t), np.ones_like(t)], 1)
    ce = np.linalg.lstsq(A, np.array(eta), rcond=None)[0]
    cp = np.linalg.lstsq(A, np.array(P), rcond=None)[0]
    return (np.hypot(ce[0], ce[1]) / a, np.hypot(cp[0], cp[1]) / a,
            np.arctan2(ce[1], ce[0]), np.arctan2(cp[1], cp[0]), w0, d)


def test_sine_maker_progressive_wave(oracle_mod):
    """Eq. 25-29 at the west end of a channel with a sponge at the east end
    (a/d = 0.005).  What the maker sends in is a wave travelling east, which
    mass conservation ties to P = c eta with c = w/k of the model's own
    linear dispersion relation c^2 = g d (1 + B (kd)^2) / (1 + (B + 1/3)
    (kd)^2) (Sec. 2.1): P in phase with eta, and an amplitude within 5 % of
    a (the ghosts carry a and Eckart's c, within a few % of the model's).
    The stages' ghost times: the steady phase converges in dt (the same to
    1e-5 rad at Courant 0.2 and 0.1), which a stage taking its ghosts one
    step off (a first-order phase error, 3e-3 rad at Courant 0.2) breaks."""
    from scipy.optimize import brentq
    amp_eta, amp_P, ph_eta, ph_P, w0, d = _sine_channel(oracle_mod, 0.2)
    km = brentq(lambda k: w0 ** 2 - G * d * k ** 2 * (1 + B * (k * d) ** 2) / (1 + (B + 1 / 3) * (k * d) ** 2),
                1e-6, 10.0)
    assert np.all(np.abs(amp_P / amp_eta / (w0 / km) - 1) <= 0.01)
    assert np.all(np.abs(np.angle(np.exp(1j * (ph_P - ph_eta)))) <= 0.01)
    assert np.all(np.abs(amp_eta - 1) <= 0.05)
    ph_half = _sine_channel(oracle_mod, 0.1)[2]
    assert np.all(np.abs(np.angle(np.exp(1j * (ph_half - ph_eta)))) <= 1e-5)


def test_boussinesq_reduces_to_nlsw_where_d_is_zero(oracle_mod):
    """Sec. 2.1: the equations reduce to the nonlinear shallow-water system
    where d = 0.  With the still-water level below the whole bed (d = 0
    everywhere) and water standing on it, the Boussinesq model steps
    exactly as the NLSW model: every dispersive and mixed term carries a
    factor d, and the rows of Eq. 23 become identity rows."""
    nx, ny = 40, 32
    z = sc.random_bed(nx, ny, 11, -1.0, -0.4, smooth=2)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    w0 = z + 0.3 + 0.1 * np.exp(-((X - 15) ** 2 + (Y - 12) ** 2) / 20.0)
    runs = []
    for model in (oracle_mod.BSNQ, oracle_mod.NLSW):
        o = oracle_mod.Oracle(z, 1.0, 1.0, 0.1 / math.sqrt(G * 0.8), model=model, K=1, ws=-5.0,
                              friction=2, fcoef=0.02, eps=1e-8)
        o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, 6)
        o.set_state(w0, 0 * z, 0 * z)
        o.step(200)
        runs.append(o.state())
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    assert np.max(np.abs(runs[0][1])) > 0


def test_linear_shoaling_on_a_slope(oracle_mod):
    """Sec. 2.1: the equations' linear shoaling is accurate for kd < 3.
    Regular waves (a/d = 0.004, T = 2 s) from a sine maker run up a 1:20
    slope from d = 1 m (kd 1.2) to 0.4 m (kd 0.68) into a sponge: the
    amplitude grows as energy-flux conservation of linear theory says,
    a2 / a1 = sqrt(Cg1 / Cg2) with Cg of w^2 = g k tanh(kd), within 3 %
    (the oracle: -1.3 %; without the depth-gradient terms of Eq. 10-11,
    -7 %; with d_x's sign flipped, +11 %)."""
    from scipy.optimize import brentq

    def k_of(w, d):
        return brentq(lambda k: w * w - G * k * math.tanh(k * d), 1e-6, 50.0)

    def cg(w, d):
        k = k_of(w, d)
        return 0.5 * w / k * (1 + 2 * k * d / math.sinh(2 * k * d))

    d1, d2, T, a, dx, slope = 1.0, 0.4, 2.0, 0.004, 0.05, 1 / 20
    w = 2 * math.pi / T
    L1, L2 = 2 * math.pi / k_of(w, d1), 2 * math.pi / k_of(w, d2)
    x1 = 2.5 * L1
    x2 = x1 + (d1 - d2) / slope
    nx = int(round((x2 + 6.0 * L2) / dx))
    x = (np.arange(nx) + 0.5) * dx
    z = np.tile(-np.where(x < x1, d1, np.where(x < x2, d1 - (x - x1) * slope, d2)), (2, 1))
    dt = 0.2 * dx / math.sqrt(G * d1)
    o = oracle_mod.Oracle(z, dx, dx, dt, K=1)
    o.set_boundary(oracle_mod.W, oracle_mod.SINE, 0, ((a, T, 0.0, 0.0),))
    o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, int(round(2.5 * L2 / dx)))
    o.set_state(0 * z, 0 * z, 0 * z)
    t_settled = x1 / (L1 / T) + (x2 - x1 + 3.5 * L2) / (L2 / T) + 8 * T
    n_total, n_fit = int(round(t_settled / dt)), int(round(3 * T / dt))
    o.step(n_total - n_fit)
    # eight gauges over a wavelength on each flat part average out the
    # partial standing wave of the slope's small reflection
    gi = [int(round((0.8 * L1 + f * L1 / 8) / dx)) for f in range(8)] + \
         [int(round((x2 + L2 + f * L2 / 8) / dx)) for f in range(8)]
    t, eta = [], []
    for n in range(n_fit):
        o.step(1)
        t.append((n_total - n_fit + n + 1) * dt)
        eta.append(o.state()[0][0, gi])
    t = np.array(t)
    A = np.stack([np.cos(w * t), np.sin(w * t), np.ones_like(t)], 1)
    ce = np.linalg.lstsq(A, np.array(eta), rcond=None)[0]
    amp = np.hypot(ce[0], ce[1])
    ratio = amp[8:].mean() / amp[:8].mean()
    assert abs(ratio / math.sqrt(cg(w, d1) / cg(w, d2)) - 1) <= 0.03


# --------------------------------------------------------------- symmetry

def test_symmetry_mirror_x(oracle_mod):
    nx, ny = 96, 4
    dx = 0.05
    x = (np.arange(nx) + 0.5) * dx
    z = np.full((ny, nx), -1.0) + 0.3 * np.exp(-((x - nx * dx / 2) / 0.8) ** 2)
    eta = 0.05 * np.exp(-((x - nx * dx / 2) / 0.5) ** 2)
    o = oracle_mod.Oracle(z, dx, dx, 0.2 * dx / math.sqrt(G), K=0)
    o.set_state(np.tile(eta, (ny, 1)), 0 * z, 0 * z)
    o.step(400)
    w, P, Q = o.state()
    scale = np.max(np.abs(w))
    assert np.max(np.abs(w - w[:, ::-1])) <= 1e-12 * scale
    assert np.max(np.abs(P + P[:, ::-1])) <= 1e-12 * max(np.max(np.abs(P)), 1e-30)
    assert np.all(Q == 0.0)
    assert np.max(np.abs(w - w[0:1])) == 0.0          # stays y-uniform


def test_symmetry_mirror_x_wet_dry(oracle_mod):
    """A parabolic basin dry at both ends with a centred hump: the shoreline
    moves up both slopes, through both branches of the positivity fix
    (Reading A-L2) and the dry clamp, and the run stays mirror-symmetric."""
    nx, ny, dx = 120, 2, 0.05
    x = (np.arange(nx) + 0.5) * dx
    xc = nx * dx / 2
    z = np.tile(-0.5 + 0.8 * ((x - xc) / xc) ** 2, (ny, 1))
    eta = np.tile(0.08 * np.exp(-((x - xc) / 0.4) ** 2), (ny, 1))
    o = oracle_mod.Oracle(z, dx, dx, 0.1 * dx / math.sqrt(G * 0.5), model=oracle_mod.NLSW, K=1, eps=1e-8)
    o.set_state(np.maximum(eta, z), 0 * z, 0 * z)
    o.step(800)
    w, P, Q = o.state()
    wet = w - z > 1e-6
    assert np.any(~wet[0, :10]) and np.any(wet[0, 10:40])    # a shoreline on the slope
    assert np.max(np.abs(w - w[:, ::-1])) <= 1e-12
    assert np.max(np.abs(P + P[:, ::-1])) <= 1e-12 * max(np.max(np.abs(P)), 1e-30)
    assert np.max(np.abs(P)) > 0


def test_symmetry_transpose_wet_dry(oracle_mod):
    """The basin of the test above with its hump off centre, run along x and
    along y: the shoreline climbs the slopes through both branches of the
    positivity fix on the y-faces as on the x-faces, and the two runs are
    transposes of each other (w, and P against Q)."""
    n, m, dx = 120, 2, 0.05
    x = (np.arange(n) + 0.5) * dx
    xc = n * dx / 2
    z1 = -0.5 + 0.8 * ((x - xc) / xc) ** 2
    eta1 = 0.08 * np.exp(-((x - 0.8 * xc) / 0.4) ** 2)

    def run(along_x):
        z = np.tile(z1, (m, 1)) if along_x else np.tile(z1[:, None], (1, m))
        eta = np.tile(eta1, (m, 1)) if along_x else np.tile(eta1[:, None], (1, m))
        o = oracle_mod.Oracle(z, dx, dx, 0.1 * dx / math.sqrt(G * 0.5), model=oracle_mod.NLSW, K=1, eps=1e-8)
        o.set_state(np.maximum(eta, z), 0 * z, 0 * z)
        o.step(800)
        return o.state(), z

    (wa, Pa, Qa), za = run(True)
    (wb, Pb, Qb), _ = run(False)
    wet = wa - za > 1e-6
    assert np.any(~wet[0, :10]) and np.any(wet[0, 10:40]) and np.any(~wet[0, -10:])
    assert np.max(np.abs(wa - wb.T)) <= 1e-12
    assert np.max(np.abs(Pa - Qb.T)) <= 1e-12 * np.max(np.abs(Pa))
    assert np.max(np.abs(Pa)) > 0 and np.all(Qa == 0.0) and np.all(Pb == 0.0)


def test_symmetry_transpose_with_sponges(oracle_mod):
    """The transpose symmetry with sponges on all four sides (Eq. 30): each
    damps w, P and Q alike, so the run stays symmetric under x <-> y with
    P <-> Q."""
    n = 48
    z = sc.random_bed(n, n, 3, -3.0, -1.5, smooth=3)
    z = 0.5 * (z + z.T)
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    eta = 0.1 * np.exp(-((X - 14) ** 2 + (Y - 32) ** 2) / 20.0)
    eta = eta + eta.T
    o = oracle_mod.Oracle(z, 0.5, 0.5, 0.05 / math.sqrt(G * 3.0), K=1)
    for side in (oracle_mod.W, oracle_mod.E, oracle_mod.S, oracle_mod.N):
        o.set_boundary(side, oracle_mod.SPONGE, 8)
    o.set_state(eta, 0 * z, 0 * z)
    o.step(300)
    w, P, Q = o.state()
    assert np.max(np.abs(w - w.T)) <= 1e-12 * np.max(np.abs(w))
    assert np.max(np.abs(P - Q.T)) <= 1e-12 * np.max(np.abs(P))


def test_sponge_profile_in_metres(oracle_mod):
    """Eq. 30 on every side, in metres: a lake raised by eps over a flat bed
    is at rest (no flux), so one step leaves w - w_s = eps gamma(D) exactly,
    with D the distance from the side's face to the cell centre and the
    layer width L = cells x spacing of that direction (dx != dy), the
    smallest gamma where layers overlap."""
    nx, ny, dx, dy, eps = 40, 30, 0.5, 0.25, 1e-3
    widths = {oracle_mod.W: 6, oracle_mod.E: 9, oracle_mod.S: 5, oracle_mod.N: 7}
    z = np.full((ny, nx), -1.0)
    o = oracle_mod.Oracle(z, dx, dy, 0.01, K=1)
    for side, wd in widths.items():
        o.set_boundary(side, oracle_mod.SPONGE, wd)
    o.set_state(np.full_like(z, eps), 0 * z, 0 * z)
    o.step(1)
    w = o.state()[0]
    xc, yc = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy
    gam = np.ones((ny, nx))
    for side, wd in widths.items():
        if side in (oracle_mod.W, oracle_mod.E):
            D, L = (xc if side == oracle_mod.W else nx * dx - xc), wd * dx
            g = np.array([oracle_mod.sponge_gamma(v, L) for v in D])[None, :]
        else:
            D, L = (yc if side == oracle_mod.S else ny * dy - yc), wd * dy
            g = np.array([oracle_mod.sponge_gamma(v, L) for v in D])[:, None]
        gam = np.minimum(gam, g)
    np.testing.assert_allclose(w, eps * gam, rtol=1e-12, atol=1e-18)
    assert (gam < 1).sum() > 0 and (gam == 1).sum() > 0


@pytest.mark.parametrize("axis", ["x", "y"])
def test_symmetry_mirror_sine_makers(oracle_mod, axis):
    """A west maker (direction 0) over a bed that varies along x, and an east
    maker (direction pi) over the mirrored bed, give mirrored runs (Eq.
    25-29): the east maker takes its depth, hence k (Eq. 29), from the cell
    beside it and its ghosts at their own x; its phase is set back by k L
    so that both makers send the same wave.  axis "y": the same with south
    and north makers over a bed that varies along y."""
    n, m, dx = 72, 6, 0.5
    s = np.arange(n)
    bed = -2.0 + 0.8 * np.exp(-((s - 60) / 8.0) ** 2) + 0.2 * np.cos(s / 5.0)
    a, T, phi = 0.01, 3.0, 0.4
    om = 2 * math.pi / T

    def run(far):
        z1 = bed[::-1] if far else bed
        z = np.tile(z1, (m, 1)) if axis == "x" else np.tile(z1[:, None], (1, m))
        o = oracle_mod.Oracle(z, dx, dx, 0.1 * dx / math.sqrt(G * 2.0), K=1)
        near_side, far_side = (oracle_mod.W, oracle_mod.E) if axis == "x" else (oracle_mod.S, oracle_mod.N)
        d = o.field("d")
        dadj = (d[0, -1] if axis == "x" else d[-1, 0]) if far else d[0, 0]     # the cell beside the maker
        k = oracle_mod.eckart_k(om, dadj, G)
        base = 0.0 if axis == "x" else math.pi / 2
        comp = (a, T, base + math.pi, phi - k * n * dx) if far else (a, T, base, phi)
        o.set_boundary(far_side if far else near_side, oracle_mod.SINE, 0, (comp,))
        o.set_state(0 * z, 0 * z, 0 * z)
        o.step(300)
        return o.state()

    wa, Pa, Qa = run(False)
    wb, Pb, Qb = run(True)
    flip = (lambda v: v[:, ::-1]) if axis == "x" else (lambda v: v[::-1, :])
    Na, Nb = (Pa, Pb) if axis == "x" else (Qa, Qb)
    assert np.max(np.abs(wa)) > 1e-3
    assert np.max(np.abs(wa - flip(wb))) <= 1e-10 * np.max(np.abs(wa))
    assert np.max(np.abs(Na + flip(Nb))) <= 1e-10 * np.max(np.abs(Na))


def test_sine_maker_beside_dry_land(oracle_mod):
    """Eq. 25-29 take the still-water depth of the cell beside the maker; in
    rows where that cell is land (d = 0) there is no depth to set k from and
    the maker sends nothing: its ghosts hold still water.  A west maker along
    a coast whose upper rows start on land 0.3 m above w_s: the run stays
    finite and the land there stays dry, with no discharge."""
    nx, ny, dx = 40, 16, 0.1
    z = np.full((ny, nx), -0.5)
    z[10:, :5] = 0.3
    o = oracle_mod.Oracle(z, dx, dx, 0.1 * dx / math.sqrt(G * 0.5), K=1)
    o.set_boundary(oracle_mod.W, oracle_mod.SINE, 0, ((0.01, 1.0, 0.0, 0.0),))
    o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, 10)
    o.set_state(0 * z, 0 * z, 0 * z)
    assert np.all(o.field("d")[10:, 0] == 0.0) and np.all(o.field("d")[:10, 0] > 0.0)
    o.step(300)
    w, P, Q = o.state()
    Bbar = o.field("Bbar")
    assert np.all(np.isfinite(w)) and np.max(np.abs(w[:10, :10])) > 1e-3     # the wave went in below
    np.testing.assert_array_equal(w[11:, :4], Bbar[11:, :4])
    assert np.all(P[11:, :4] == 0.0) and np.all(Q[11:, :4] == 0.0)


def test_symmetry_transpose_sine_makers(oracle_mod):
    """A west maker at direction 0 beside a south wall, and the transposed
    set-up, a south maker at direction pi/2 beside a west wall (Eq. 25-29,
    sponges on the far sides), give transposed runs (x <-> y, P <-> Q): the
    y-sides' maker ghosts, their discharge along y and the y-lines' maker
    rows against the x-sides' (corner ghosts transpose too here, as each
    corner touches one maker)."""
    n = 64
    z = sc.random_bed(n, n, 3, -3.0, -1.5, smooth=3)
    z = 0.5 * (z + z.T)

    def run(west):
        o = oracle_mod.Oracle(z, 1.0, 1.0, 0.1 / math.sqrt(G * 3.0), K=1)
        o.set_boundary(oracle_mod.W if west else oracle_mod.S, oracle_mod.SINE, 0,
                       ((0.02, 6.0, 0.0 if west else math.pi / 2, 0.3),))
        o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, 10)
        o.set_boundary(oracle_mod.N, oracle_mod.SPONGE, 10)
        o.set_state(0 * z, 0 * z, 0 * z)
        o.step(600)
        return o.state()

    wa, Pa, Qa = run(True)
    wb, Pb, Qb = run(False)
    scale = np.max(np.abs(Pa))
    assert np.max(np.abs(wa)) > 0.01
    assert np.max(np.abs(wa - wb.T)) <= 1e-12 * np.max(np.abs(wa))
    assert np.max(np.abs(Pa - Qb.T)) <= 1e-12 * scale and np.max(np.abs(Qa - Pb.T)) <= 1e-12 * scale


def test_symmetry_transpose_solitons(oracle_mod):
    """A solitary wave heading along x (direction 0) and the transposed one
    heading along y (pi/2) in a walled square basin (Eq. 33-36) give
    transposed runs: the wave's discharge along its direction in y."""
    n, dx, d = 64, 0.5, 1.0
    z = np.full((n, n), -d)

    def run(along_x):
        o = oracle_mod.Oracle(z, dx, dx, 0.1 * dx / math.sqrt(G * d), K=1)
        o.set_state(0 * z, 0 * z, 0 * z)
        if along_x:
            o.add_solitary(0.1, 0.0, 9.0, 17.0)
        else:
            o.add_solitary(0.1, math.pi / 2, 17.0, 9.0)
        o.step(200)
        return o.state()

    wa, Pa, Qa = run(True)
    wb, Pb, Qb = run(False)
    scale = np.max(np.abs(Pa))
    assert np.max(np.abs(wa)) > 0.05
    assert np.max(np.abs(wa - wb.T)) <= 1e-12 * np.max(np.abs(wa))
    assert np.max(np.abs(Pa - Qb.T)) <= 1e-12 * scale and np.max(np.abs(Qa - Pb.T)) <= 1e-12 * scale


def test_symmetry_transpose(oracle_mod):
    n = 48
    z = sc.random_bed(n, n, 3, -3.0, -1.5, smooth=3)
    z = 0.5 * (z + z.T)
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    eta = 0.1 * np.exp(-((X - 18) ** 2 + (Y - 30) ** 2) / 20.0)
    eta = eta + eta.T
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.1 / math.sqrt(G * 3.0), K=1)
    o.set_state(eta, 0 * z, 0 * z)
    o.step(300)
    w, P, Q = o.state()
    assert np.max(np.abs(w - w.T)) <= 1e-12 * np.max(np.abs(w))
    assert np.max(np.abs(P - Q.T)) <= 1e-12 * np.max(np.abs(P))


# -------------------------------------------------------------- stability

def _growth(oracle_mod, cr, model, K, depth=9.0, dx=1.0, n=32, steps=1500):
    z = np.full((n, n), -depth)
    rng = np.random.default_rng(0)
    o = oracle_mod.Oracle(z, dx, dx, cr * dx / math.sqrt(G * depth), model=model, K=K)
    o.set_state(1e-6 * rng.standard_normal((n, n)), 0 * z, 0 * z)
    o.step(steps)
    P = o.state()[1]
    return float(np.max(np.abs(P))) if np.all(np.isfinite(P)) else math.inf


def test_stability_ab3_real_axis_bound(oracle_mod):
    """KP07 damps a 2-D checkerboard at rate -4c/dx; AB3 (Eq. 15-17) is
    stable on the negative real axis only down to -6/11, so the NLSW step
    is stable for Courant < 3/22 = 0.136 and not above."""
    assert _growth(oracle_mod, 0.13, oracle_mod.NLSW, 0) < 1e-4
    assert _growth(oracle_mod, 0.145, oracle_mod.NLSW, 0) > 1.0


def test_stability_corrector_parity(oracle_mod):
    """With depth/dx >> 1 the explicitly extrapolated mixed terms (F*, G*)
    grow for K = 0 and even K and are bounded for odd K."""
    assert _growth(oracle_mod, 0.1, oracle_mod.BSNQ, 0, steps=600) > 1.0
    assert _growth(oracle_mod, 0.1, oracle_mod.BSNQ, 1) < 1e-4
    assert _growth(oracle_mod, 0.1, oracle_mod.BSNQ, 2, steps=600) > 1.0
    assert _growth(oracle_mod, 0.1, oracle_mod.BSNQ, 3) < 1e-4


# ------------------------------------------------------------ host logic

def test_set_state_clamps_to_bed(oracle_mod):
    z = np.array([[-1.0, -1.0, 0.5, 1.0]] * 3)
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.01)
    o.set_state(np.zeros_like(z), np.ones_like(z), np.ones_like(z))
    w, P, Q = o.state()
    Bb = o.field("Bbar")
    assert np.all(w >= Bb)
    dry = (w - Bb) <= 0
    assert dry.any()
    assert np.all(P[dry] == 0) and np.all(Q[dry] == 0)
    assert np.all(P[~dry] == 1)


def test_add_solitary_rejects_dry_crest(oracle_mod):
    z = np.array([[-1.0] * 4 + [1.0] * 4] * 3)
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.01)
    with pytest.raises(ValueError):
        o.add_solitary(0.1, 0.0, 7.5, 1.5)
    o.add_solitary(0.1, 0.0, 1.5, 1.5)


def test_gauge_ring(oracle_mod):
    s = sc.soliton_channel(steps=0)
    o = oracle_from(s)
    o.set_gauges([(10, 5), (200, 16)], log_every=3, capacity=4)
    o.step(20)                 # records at steps 3,6,...,18 -> 6, keeps last 4
    rec = o.read_gauges(10)
    assert rec.shape == (4, 2)
    o2 = oracle_from(s)
    etas = []
    for n in range(1, 21):
        o2.step(1)
        if n % 3 == 0:
            w = o2.state()[0]
            etas.append([w[5, 10], w[16, 200]])
    np.testing.assert_array_equal(rec, np.array(etas[-4:]))
    assert o.read_gauges(10).shape == (0, 2)


def test_gauges_record_eta_about_the_still_water_level(oracle_mod):
    """Gauges record the free surface's elevation eta = w - w_s (Sec. 2.1's
    eta over the still-water level): still water at w_s = 0.3 m over a
    random bed records zero at every gauge, and a raised lake records its
    rise."""
    nx, ny = 40, 30
    rng = np.random.default_rng(5)
    z = -1.0 - 0.5 * rng.random((ny, nx))
    for rise in (0.0, 0.02):
        o = oracle_mod.Oracle(z, 1.0, 1.0, 0.05, K=1, ws=0.3)
        o.set_state(np.full_like(z, 0.3 + rise), 0 * z, 0 * z)
        o.set_gauges([(3, 4), (20, 15), (37, 27)], log_every=1, capacity=8)
        o.step(5)
        rec = o.read_gauges(8)
        assert rec.shape == (5, 3)
        np.testing.assert_allclose(rec, rise, rtol=0, atol=1e-12)


def test_dry_land_holds_no_water_and_no_discharge(oracle_mod):
    """A 0.2 m hump of water runs up a steep planar beach (1:2) and back
    (Boussinesq, K = 1), far enough that the dry clamp of Reading A-D1 has
    to act.  Checked every 50 steps: the surface never lies below the bed;
    wherever the depth is zero the discharges are zero; and the flux form
    conserves mass (Eq. 1, walls all round), so the mass changes by exactly
    what the clamp reports it added.  Land the wave never reaches keeps w
    equal to its bed, which on a plane is the input z away from the mirrored
    edge cells and the beach's toe."""
    nx, ny, dx = 160, 4, 0.05
    x = (np.arange(nx) + 0.5) * dx
    z = np.tile(-0.4 + 0.5 * np.maximum(x - 2.5, 0.0), (ny, 1))     # shoreline at x = 3.3 m
    eta = 0.2 * np.exp(-((x - 1.5) / 0.3) ** 2)
    o = oracle_mod.Oracle(z, dx, dx, 0.2 * dx / math.sqrt(G * 0.6), K=1)
    o.set_state(np.tile(eta, (ny, 1)), 0 * z, 0 * z)     # land: w clamped up to its bed
    Bbar = o.field("Bbar")
    plane = (np.abs(x - 2.5) > 2 * dx) & (np.arange(nx) > 0) & (np.arange(nx) < nx - 1)
    np.testing.assert_allclose(Bbar[:, plane], z[:, plane], rtol=0, atol=1e-14)
    m0 = o.mass()
    for _ in range(20):
        o.step(50)
        w, P, Q = o.state()
        assert np.all(w >= Bbar)
        dry = w - Bbar <= 0.0
        assert dry.any()
        assert np.all(P[dry] == 0.0) and np.all(Q[dry] == 0.0)
        assert o.mass() - o.clamp_mass() == pytest.approx(m0, rel=1e-12)
    assert o.clamp_mass() > 0.0                  # the clamp acted
    far = plane & (x > 5.5)
    np.testing.assert_allclose(w[:, far], z[:, far], rtol=0, atol=1e-14)


def test_runup_tracking_standing_mode(oracle_mod):
    """Run-up tracking (Sec. 4.1, 4.3) keeps the highest w seen: over half a
    period of the 1-D standing mode eta = a cos(kx) cos(wt) it must be
    |a cos(kx)| everywhere (the initial and the final state each give only
    half of the cells), within the scheme's amplitude error."""
    d, kd, cpl = 1.0, 1.0, 64
    k = kd / d
    dx = 2 * math.pi / k / cpl
    x = (np.arange(cpl) + 0.5) * dx
    a = 1e-4 * d
    eta = np.tile(a * np.cos(k * x), (2, 1))
    z = np.full((2, cpl), -d)
    dt = 0.2 * dx / math.sqrt(G * d)
    o = oracle_mod.Oracle(z, dx, dx, dt)
    o.set_state(eta, 0 * z, 0 * z)
    o.runup_enable(0.5 * d)
    first = o.runup()[0].copy()
    np.testing.assert_array_equal(first, eta[0])           # starts from the state
    T = 2 * math.pi / _omega(k, d)
    o.step(int(round(0.5 * T / dt)))
    m = o.runup()[0]
    last = o.state()[0][0]
    assert np.max(np.abs(m - np.abs(a * np.cos(k * x)))) <= 0.03 * a
    assert np.all(m >= np.maximum(first, last))            # never below what it saw
    assert np.max(np.abs(m - last)) > 0.5 * a              # not the last state


def test_runup_tracking_threshold_and_dry_land(oracle_mod):
    """Cells never deeper than the threshold keep -inf: dry land behind a
    lake, the whole lake once the threshold exceeds its depth, and a lake
    exactly as deep as the threshold."""
    z = np.full((4, 12), -0.05)
    z[:, 8:] = 0.4
    o = oracle_mod.Oracle(z, 1.0, 1.0, 0.01)
    o.runup_enable(0.01)
    o.step(5)
    m = o.runup()
    # column 7's cell bed (the mean of its corners, which average in the
    # land) is above w_s, so it is dry too
    assert np.all(np.isneginf(m[:, 7:]))
    np.testing.assert_allclose(m[:, :7], 0.0, atol=1e-14)   # lake at rest: w = w_s
    o.runup_enable(0.06)
    o.step(2)
    assert np.all(np.isneginf(o.runup()))
    # the threshold is strict: a lake exactly delta deep (a power of two, so
    # w - Bbar = delta exactly, and exactly at rest) never exceeded it
    zf = np.full((4, 12), -0.0625)
    of = oracle_mod.Oracle(zf, 1.0, 1.0, 0.01)
    of.runup_enable(0.0625)
    of.step(3)
    assert np.all(np.isneginf(of.runup()))
    of.runup_enable(0.0624)
    of.step(1)
    np.testing.assert_array_equal(of.runup(), 0.0)


def _uniform_flow_states(oracle_mod, K, nsteps, dt=0.01, f=0.5, P0=0.5):
    """P after 0..nsteps steps in the middle of a uniform 1 m deep flow under
    quadratic friction: away from the walls the step is the ODE update of
    P' = F(P) = -f P |P| (h = 1, so Eq. 14's k(h) = 1)."""
    nx, ny, dx = 400, 2, 0.1
    z = np.full((ny, nx), -1.0)
    out = []
    for n in range(nsteps + 1):
        o = oracle_mod.Oracle(z, dx, dx, dt, model=oracle_mod.NLSW, friction=1, fcoef=f, K=K)
        o.set_state(0 * z, P0 + 0 * z, 0 * z)
        o.step(n)
        out.append(o.state()[1][0, nx // 2])
    return out


@pytest.mark.parametrize("K", [0, 1, 3])
def test_time_stepping_formulas_step_by_step(oracle_mod, K):
    """Sec. 2.3, one step at a time on the friction ODE: steps 1 and 2 are
    forward Euler; step 3 is the AB3 predictor (Eq. 15-17, weights 23, -16,
    5 over 12) and, with K corrector iterations, K applications of the AM4
    corrector (Eq. 18-20, weights 9, 19, -5, 1 over 24) starting from the
    predicted value.  Each checked against the formula with the oracle's
    own previous states, to rounding."""
    dt, f = 0.01, 0.5
    F = lambda P: -f * P * abs(P)
    P = _uniform_flow_states(oracle_mod, K, 3, dt=dt, f=f)
    assert P[1] == pytest.approx(P[0] + dt * F(P[0]), rel=1e-14, abs=0)
    assert P[2] == pytest.approx(P[1] + dt * F(P[1]), rel=1e-14, abs=0)
    y = P[2] + dt / 12 * (23 * F(P[2]) - 16 * F(P[1]) + 5 * F(P[0]))
    for _ in range(K):
        y = P[2] + dt / 24 * (9 * F(y) + 19 * F(P[2]) - 5 * F(P[1]) + F(P[0]))
    assert P[3] == pytest.approx(y, rel=1e-14, abs=0)
    if K >= 1:   # and not the predictor alone: the corrector moved the value
        ab3 = P[2] + dt / 12 * (23 * F(P[2]) - 16 * F(P[1]) + 5 * F(P[0]))
        assert abs(P[3] - ab3) > 1e-9


# ------------------------------------------------ isotropy and corner ghosts

def _radial_anisotropy(oracle_mod, dx, R=4.0, dc=0.5, slope=0.3, sig=0.5, a=0.005, T=0.7):
    """A Gaussian hump at rest over a round shoal whose depth grows with the
    radius (d = dc + slope sqrt(r^2 + 1/4)), on a square grid centred on one
    cell, walls far enough that the wave has not reached them at T.  Returns
    (mismatch between eta along the diagonals and eta along the axes at the
    same radius, relative L2; the largest spread between the four axes and
    between the four diagonals, relative)."""
    from scipy.interpolate import CubicSpline
    n = int(round(2 * R / dx)) | 1
    c = n // 2
    x = (np.arange(n) - c) * dx
    X, Y = np.meshgrid(x, x)
    r = np.hypot(X, Y)
    d = dc + slope * np.sqrt(r ** 2 + 0.25)
    dt = 0.2 * dx / math.sqrt(G * d.max())
    o = oracle_mod.Oracle(-d, dx, dx, dt, K=1, eps=1e-8)
    o.set_state(a * np.exp(-r ** 2 / sig ** 2), 0 * r, 0 * r)
    o.step(int(round(T / dt)))
    w = o.state()[0]
    k = np.arange(c + 1)
    axes = [w[c, c + k], w[c, c - k], w[c + k, c], w[c - k, c]]
    diags = [w[c + k, c + k], w[c - k, c - k], w[c + k, c - k], w[c - k, c + k]]
    top = np.abs(axes[0]).max()
    spread = max(max(np.abs(v - axes[0]).max() for v in axes), max(np.abs(v - diags[0]).max() for v in diags)) / top
    ra, rd = k * dx, k * dx * math.sqrt(2.0)
    along = CubicSpline(ra, axes[0])
    m = rd <= 0.9 * ra[-1]
    mismatch = np.linalg.norm(diags[0][m] - along(rd[m])) / np.linalg.norm(along(rd[m]))
    return mismatch, spread


def test_isotropy_over_a_round_shoal(oracle_mod):
    """The equations are isotropic (Eq. 2-3, 7-13): with M = (P, Q) the
    depth-gradient terms of the momentum equations are
    d [grad d (div M) + (grad M)^T grad d] / 6 under the time derivative (the
    1/3 of Eq. 7 and the two 1/6 of Eq. 12), and B g d^2 [grad d lap eta +
    hess(eta) grad d] (Eq. 10-11).  So a radially symmetric problem has a
    radially symmetric solution, and on the grid eta along the diagonals must
    approach eta along the axes as the grid is refined.  On a round shoal
    every depth-gradient term of F*, G* and of Eq. 10-11 is active: dropping
    one, or weighting it 1/3 instead of 1/6, leaves an anisotropy that does
    not shrink with the grid (measured: 0.013-0.026 at dx = 0.025, where this
    oracle gives 0.004, converging from 0.008 at dx = 0.05).  The four axes
    (and the four diagonals) agree to rounding by the grid's own symmetry."""
    coarse, s1 = _radial_anisotropy(oracle_mod, 0.05)
    fine, s2 = _radial_anisotropy(oracle_mod, 0.025)
    assert s1 <= 1e-12 and s2 <= 1e-12
    assert fine <= 6.5e-3, (coarse, fine)
    assert fine <= 0.65 * coarse, (coarse, fine)


def test_corner_ghost_of_a_maker_beside_a_wall_by_embedding(oracle_mod):
    """Corner ghosts (Reading A-B5) where a sine maker meets a wall.  The
    face-centred wall at y = 0 (Reading A-B1) is an even mirror: a run on
    the upper half with a south wall is exactly the upper half of a run on a
    domain twice as high whose bed, state and west maker are even about the
    middle (two components at +-theta, phased so that their sum is even:
    Eq. 25-28).  The corner ghost at (-1, -1) that the half run builds (the
    mirror of the maker's ghost beside it, Q negated) is what the doubled run
    holds there; cell (0, 0)'s mixed derivatives read it."""
    nx, m, dx, d0, T, a, th = 64, 32, 0.25, 1.0, 3.0, 0.01, 0.5
    rng = np.random.default_rng(21)
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(m) + 0.5) * dx)
    # flat beside the maker (its wave number follows the depth there), a
    # shoal, a slope and noise beyond
    z = -d0 + (0.3 * np.exp(-((X - 9.0) ** 2 + (Y - 3.0) ** 2) / 4.0) + 0.02 * (X - 3.0)
               + 0.05 * rng.standard_normal(X.shape)) * (X > 3.0)
    z_big = np.vstack([z[::-1], z])
    dt = 0.1 * dx / math.sqrt(G * d0)
    k = oracle_mod.eckart_k(2 * math.pi / T, d0)
    ymid = m * dx

    def run(zz, comps, south):
        o = oracle_mod.Oracle(zz, dx, dx, dt, K=1, eps=1e-8)
        o.set_boundary(oracle_mod.W, oracle_mod.SINE, 0, comps)
        o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, 12)
        o.set_boundary(oracle_mod.S, south)
        o.set_state(0 * zz, 0 * zz, 0 * zz)
        o.step(400)
        return o.state()

    half = run(z, ((a, T, th, 0.0), (a, T, -th, 0.0)), oracle_mod.SOLID)
    big = run(z_big, ((a, T, th, k * math.sin(th) * ymid), (a, T, -th, -k * math.sin(th) * ymid)),
              oracle_mod.SOLID)
    wh, Ph, Qh = half
    wb, Pb, Qb = (v[m:] for v in big)
    assert np.max(np.abs(wh)) > 0.005
    scale = np.max(np.abs(Ph))
    assert np.max(np.abs(wh - wb)) <= 1e-11 * np.max(np.abs(wh))
    assert np.max(np.abs(Ph - Pb)) <= 1e-11 * scale and np.max(np.abs(Qh - Qb)) <= 1e-11 * scale


def test_corner_ghosts_where_two_makers_meet(oracle_mod):
    """Corner ghosts (Reading A-B5) where two sine makers meet: west and
    south makers sending the same plane wave at 45 degrees over a flat bed
    (Eq. 25-28), sponges east and north.  Both makers' formulas give the
    same value at the corner ghost, the plane wave there.  The run is its
    own transpose (x <-> y, P <-> Q) up to 1e-4: at the far corners, inside
    the sponges, a maker meets a sponge side, and there the x-sides-first
    composition gives the mirror of the west maker's ghost at the north-west
    corner but the south maker's own value at the south-east one (measured
    2.6e-5 of the amplitude).  The complex amplitude of eta near
    the corner follows the plane wave: the phase step between neighbouring
    cells and the amplitude at the corner cell stay within a few per cent of
    the values far from the corner (what differs is the makers' boundary
    layer, from Eckart's wave number against the model's).  A corner ghost
    left unset (or set to still water) breaks both by 10-20 %: cell (0, 0)'s
    mixed derivatives (Eq. 10-13) read it."""
    n, dx, d0, T, a, th = 160, 0.05, 0.5, 1.5, 0.002, math.pi / 4
    z = np.full((n, n), -d0)
    dt = 0.2 * dx / math.sqrt(G * d0)
    o = oracle_mod.Oracle(z, dx, dx, dt, K=1, eps=1e-8)
    comps = ((a, T, th, 0.0),)
    o.set_boundary(oracle_mod.W, oracle_mod.SINE, 0, comps)
    o.set_boundary(oracle_mod.S, oracle_mod.SINE, 0, comps)
    o.set_boundary(oracle_mod.E, oracle_mod.SPONGE, 40)
    o.set_boundary(oracle_mod.N, oracle_mod.SPONGE, 40)
    m = 12
    steps = int(round(8 * T / dt))
    o.set_gauges([(i, j) for j in range(m) for i in range(m)], 1, steps)
    o.step(steps)
    w, P, Q = o.state()
    assert np.max(np.abs(w - w.T)) <= 1e-4 * np.max(np.abs(w))
    assert np.max(np.abs(P - Q.T)) <= 1e-4 * np.max(np.abs(P))
    rec = o.read_gauges(steps)
    t = dt * np.arange(1, steps + 1)
    last = t > 5 * T
    om = 2 * math.pi / T
    M = np.stack([np.sin(om * t[last]), np.cos(om * t[last]), np.ones(last.sum())], 1)
    coef = np.linalg.lstsq(M, rec[last], rcond=None)[0]
    A = (coef[0] + 1j * coef[1]).reshape(m, m)        # A[j, i]
    rx, ry = A[:, 1:] / A[:, :-1], A[1:, :] / A[:-1, :]
    far_rx, far_ry = rx[6:, 6:].mean(), ry[6:, 6:].mean()
    assert np.abs(rx[6:, 6:] - far_rx).max() <= 0.01          # a plane wave far from the corner
    assert np.abs(rx[:3, :3] - far_rx).max() <= 0.05 and np.abs(ry[:3, :3] - far_ry).max() <= 0.05
    assert abs(A[0, 0]) >= 0.87 * np.abs(A[6:, 6:]).mean()
