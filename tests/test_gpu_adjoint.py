"""Discrete adjoint (cel_adjoint_gauge_misfit) vs FP64 finite differences of
the oracle and vs the FP64 tangent-linear oracle (the oracle's own source on
dual numbers), for the gradients with respect to the initial w and the bed z.

The loss is the gauge misfit L = 1/2 sum over steps and gauges of
(eta - obs)^2.  The step is piecewise smooth: the generalized minmod, the
wave-speed bounds and the wet/dry clamps switch branches, and a state at
rest sits on a minmod kink in every cell (a directional derivative there is
not linear in the direction), so finite differences are compared where the
state is away from kinks: a tilted free surface with a steady discharge
(every slope of one sign, the limiter on one branch with a 30 % margin),
quadratic friction, a sponge, a sine maker, walls, the Euler start-up and
the AB3 history.  There <dL/dw0, v> from the GPU adjoint must match the
oracle's central difference (L(w0 + e v) - L(w0 - e v)) / 2e within 1e-3
relative for seeded smooth directions v, and <dL/dz, v> the difference of
L(z + e v) and L(z - e v) at fixed w0.  Shallow water without a sponge or a
wave maker is unchanged when w and z move up together, so there
sum(dL/dw0 + dL/dz) equals the summed misfit exactly, dry land included.
A beach with dry land and a moving
shoreline checks the rest: checkpoint spacing changes nothing, the loss and
the gauge records equal the oracle's, land far from the water gets a zero
gradient; FP32 agrees with FP64 on the kink-free state.
"""
import math

import numpy as np
import pytest

from tests.helpers import oracle_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _scenario(nsteps=60):
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx = 56, 40, 0.1
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    z = np.maximum(-0.5, (X - 4.2) * 0.25) + 0.05 * np.exp(-((X - 2.0) ** 2 + (Y - 2.0) ** 2) / 0.3)
    d0 = 0.5
    dt = 0.1 * dx / math.sqrt(9.81 * d0)
    s = sc.flat_basin(nx, ny, dx, d0, dt, model=1, K=0, friction=2, fcoef=0.02, eps=1e-8)
    s.z = z
    s.sides[sc.W] = sc.Side(sc.SPONGE, 6)
    w0 = np.maximum(z, 0.08 * np.exp(-((X - 2.6) ** 2 + (Y - 1.6) ** 2) / 0.15))
    s.w0 = w0
    s.steps = nsteps
    rng = np.random.default_rng(11)
    gauges = [(int(rng.integers(8, 40)), int(rng.integers(3, ny - 3))) for _ in range(6)]
    return s, gauges


def _oracle_loss(s, w0, gauges, obs):
    o = oracle_from(s)
    w, P, Q = s.initial_state()
    o.set_state(w0, P, Q)
    o.set_gauges(gauges, 1, s.steps)
    o.step(s.steps)
    eta = o.read_gauges(s.steps)
    return 0.5 * float(np.sum((eta - obs) ** 2)), eta


def _gpu_gradient(s, gauges, obs, prec="f64", ckpt=7, bed=False):
    from paper_1611_05984_gb300 import celeris
    dtype = torch.float64 if prec == "f64" else torch.float32
    g = celeris.from_scenario(s, dtype=dtype)
    out = celeris.gauge_misfit_gradient(g, s.steps, gauges, torch.as_tensor(obs, dtype=dtype), ckpt, bed=bed)
    loss, eta, grad = out[:3]
    res = (loss, eta.double().cpu().numpy(), grad.double().cpu().numpy(), g)
    return res + (out[3].double().cpu().numpy(),) if bed else res


def _tilted(nsteps=15):
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx, d0 = 48, 36, 0.1, 0.5
    dt = 0.1 * dx / math.sqrt(9.81 * d0)
    s = sc.flat_basin(nx, ny, dx, d0, dt, model=1, K=0, friction=1, fcoef=0.01, eps=1e-8)
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    s.w0 = 0.04 * X / (nx * dx) + 0.02 * Y / (ny * dx) + 0.002 * np.exp(-((X - 2.0) ** 2 + (Y - 1.5) ** 2) / 0.5)
    s.P0 = 0.02 + 0.01 * X / (nx * dx)
    s.Q0 = 0.01 + 0.005 * Y / (ny * dx)
    s.sides[sc.E] = sc.Side(sc.SPONGE, 6)
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.01, 2.0, 0.2, 0.3),))
    s.steps = nsteps
    rng = np.random.default_rng(7)
    gauges = [(int(rng.integers(4, nx - 4)), int(rng.integers(3, ny - 3))) for _ in range(6)]
    return s, gauges, X, Y


def _oracle_loss_state(s, w0, gauges, obs):
    o = oracle_from(s)
    _, P, Q = s.initial_state()
    o.set_state(w0, P, Q)
    o.set_gauges(gauges, 1, s.steps)
    o.step(s.steps)
    return 0.5 * float(np.sum((o.read_gauges(s.steps) - obs) ** 2))


def test_adjoint_matches_oracle_finite_differences_away_from_kinks():
    s, gauges, X, Y = _tilted()
    rng = np.random.default_rng(3)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, eta, grad, g = _gpu_gradient(s, gauges, obs, ckpt=4)
    assert abs(loss - _oracle_loss_state(s, s.w0, gauges, obs)) <= 1e-9 * loss
    assert g.time()[1] == s.steps                      # left after the last step
    eps = 1e-5
    errs = []
    for _ in range(8):
        v = np.zeros_like(X)
        for _ in range(3):
            cx, cy = rng.uniform(0.5, 4.3), rng.uniform(0.5, 3.1)
            v += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(0.1, 0.4))
        v *= 1e-3                                       # the perturbed field stays monotone
        fd = (_oracle_loss_state(s, s.w0 + eps * v, gauges, obs)
              - _oracle_loss_state(s, s.w0 - eps * v, gauges, obs)) / (2 * eps)
        ad = float(np.sum(grad * v))
        errs.append(abs(ad - fd) / abs(fd))
    assert max(errs) <= 1e-3, errs


def test_adjoint_beach_loss_and_records_match_oracle():
    s, gauges = _scenario()
    rng = np.random.default_rng(3)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, eta, grad, g = _gpu_gradient(s, gauges, obs)
    lo, eta_o = _oracle_loss(s, s.w0, gauges, obs)
    assert abs(loss - lo) <= 1e-9 * abs(lo)
    np.testing.assert_allclose(eta, eta_o, rtol=0, atol=1e-11)
    bed = g.field("Bbar").double().cpu().numpy()
    # land a dozen cells behind the shoreline: every face there has dry cells
    # on both sides and a zero flux whatever w, so the gradient is exactly 0
    land = s.z > 0.3
    assert np.any(land) and np.all(grad[land] == 0.0)
    assert np.any(grad[(s.w0 - bed) > 0.1] != 0.0)


def test_adjoint_checkpoint_spacing_and_fp32():
    s, gauges = _scenario(nsteps=40)
    obs = np.zeros((s.steps, len(gauges)))
    _, _, g7, _ = _gpu_gradient(s, gauges, obs, ckpt=7)
    _, _, g40, _ = _gpu_gradient(s, gauges, obs, ckpt=40)
    _, _, g1, _ = _gpu_gradient(s, gauges, obs, ckpt=1)
    _, _, g0, _ = _gpu_gradient(s, gauges, obs, ckpt=0)   # every step kept, no recomputation
    n = np.linalg.norm(g40)
    assert n > 0
    assert np.linalg.norm(g7 - g40) <= 1e-10 * n
    assert np.linalg.norm(g1 - g40) <= 1e-10 * n
    assert np.linalg.norm(g0 - g40) <= 1e-10 * n
    # FP32 against FP64 where the branches are robust (on the beach the
    # hump's exponential tail flushes to zero in FP32 and sits on another,
    # equally valid branch of the limiter's kink)
    t, tg, _, _ = _tilted()
    obs_t = np.zeros((t.steps, len(tg)))
    _, _, h64, _ = _gpu_gradient(t, tg, obs_t, ckpt=4)
    _, _, h32, _ = _gpu_gradient(t, tg, obs_t, prec="f32", ckpt=4)
    # measured 2.4e-3: FP32 reciprocals and square roots are the fast ~2 ulp
    # ones, and the gradient is more sensitive to rounding than the state
    assert np.linalg.norm(h32 - h64) <= 5e-3 * np.linalg.norm(h64)
    b, bg, _, _ = _tilted_bed(0, 1, 2)
    obs_b = np.zeros((b.steps, len(bg)))
    _, _, _, _, z64 = _gpu_gradient(b, bg, obs_b, ckpt=4, bed=True)
    _, _, _, _, z32 = _gpu_gradient(b, bg, obs_b, prec="f32", ckpt=4, bed=True)
    assert np.linalg.norm(z32 - z64) <= 1e-2 * np.linalg.norm(z64)


def test_autograd_function_and_rejections():
    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc
    s, gauges = _scenario(nsteps=20)
    obs = np.zeros((s.steps, len(gauges)))
    g = celeris.from_scenario(s, dtype=torch.float64)
    w0 = torch.tensor(s.w0, dtype=torch.float64, device="cuda", requires_grad=True)
    zero = torch.zeros_like(w0).detach()
    L = celeris.gauge_misfit(w0, g, zero, zero, s.steps, gauges, torch.as_tensor(obs), 5)
    L.backward()
    _, _, ref, _ = _gpu_gradient(s, gauges, obs, ckpt=5)
    bed = g.field("Bbar").double().cpu().numpy()
    want = np.where(s.w0 > bed, ref, 0.0)
    np.testing.assert_allclose(w0.grad.cpu().numpy(), want, rtol=1e-9, atol=1e-14)
    # with the bed as a second input
    w1 = torch.tensor(s.w0, dtype=torch.float64, device="cuda", requires_grad=True)
    zt = torch.tensor(s.z, dtype=torch.float64, device="cuda", requires_grad=True)
    L2 = celeris.gauge_misfit(w1, g, zero, zero, s.steps, gauges, torch.as_tensor(obs), 5, z=zt)
    (3.0 * L2).backward()
    _, _, _, _, refz = _gpu_gradient(s, gauges, obs, ckpt=5, bed=True)
    np.testing.assert_allclose(zt.grad.cpu().numpy(), 3.0 * refz, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(w1.grad.cpu().numpy(), 3.0 * want, rtol=1e-9, atol=1e-14)
    # the clamp's derivative by itself (cel_adjoint_input_gradient): 1 above
    # the cell bed, 0 below it and at a tie (the one-sided derivative)
    bed_t = torch.as_tensor(bed, device="cuda")
    w_in = bed_t + torch.tensor([-0.5, 0.0, 0.25], dtype=torch.float64, device="cuda").repeat(bed.size)[:bed.size] \
        .reshape(bed.shape)
    gin = torch.arange(1, bed.size + 1, dtype=torch.float64, device="cuda").reshape(bed.shape)
    gout = gin.clone()
    assert g.L.cel_adjoint_input_gradient(g._h, w_in.data_ptr(), gout.data_ptr()) == 0
    torch.cuda.synchronize()
    assert torch.equal(gout, torch.where(w_in > bed_t, gin, torch.zeros_like(gin)))
    assert g.L.cel_adjoint_input_gradient(g._h, None, gout.data_ptr()) == 1
    b = celeris.from_scenario(sc.beach(nx=64, ny=48, sponge=8), dtype=torch.float64)
    with pytest.raises(celeris.CelerisError):                       # a gauge off the grid
        celeris.gauge_misfit_gradient(b, 5, [(64, 3)], torch.zeros((5, 1), dtype=torch.float64))
    b.step(1)
    with pytest.raises(celeris.CelerisError):                       # the history is not fresh
        celeris.gauge_misfit_gradient(b, 5, [(6, 3)], torch.zeros((5, 1), dtype=torch.float64))


def _tilted_bsnq(model, nsteps=12, K=0):
    """Boussinesq-ready kink-free state: a tilted surface and discharge with
    cubic terms and a short ripple (wavelength 8 cells, depth/dx = 1, so the
    dispersive and mixed terms matter and K = 0 is stable), every slope of
    one sign."""
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx, d0 = 48, 36, 0.5, 0.5
    dt = 0.1 * dx / math.sqrt(9.81 * d0)
    s = sc.flat_basin(nx, ny, dx, d0, dt, model=model, K=K, friction=1, fcoef=0.01, eps=1e-8)
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    xs, ys = X / (nx * dx), Y / (ny * dx)
    s.w0 = 0.04 * xs + 0.03 * xs ** 3 + 0.02 * ys + 0.015 * ys ** 3 + 0.004 * xs * ys \
        + 3e-4 * np.sin(2 * math.pi * X / 4.0) * np.sin(2 * math.pi * Y / 4.0)
    s.P0 = 0.02 + 0.01 * xs + 0.01 * xs ** 3
    s.Q0 = 0.01 + 0.005 * ys + 0.006 * ys ** 3
    s.sides[sc.E] = sc.Side(sc.SPONGE, 6)
    s.steps = nsteps
    rng = np.random.default_rng(9)
    gauges = [(int(rng.integers(4, nx - 4)), int(rng.integers(3, ny - 3))) for _ in range(6)]
    return s, gauges, X, Y


def test_adjoint_boussinesq_matches_oracle_away_from_kinks():
    """The Boussinesq model: the transposed line solves, the dispersive eta
    terms and F*, G* (with their AB3 history) join the reverse.  Checked as a
    whole, and the dispersive part alone (Boussinesq minus shallow-water
    gradient against the same difference of finite differences)."""
    sb, gauges, X, Y = _tilted_bsnq(0)
    sn, _, _, _ = _tilted_bsnq(1)
    rng = np.random.default_rng(4)
    obs = 0.01 * rng.standard_normal((sb.steps, len(gauges)))
    lb, _, gb, _ = _gpu_gradient(sb, gauges, obs, ckpt=5)
    ln, _, gn, _ = _gpu_gradient(sn, gauges, obs, ckpt=5)
    assert abs(lb - _oracle_loss_state(sb, sb.w0, gauges, obs)) <= 1e-9 * lb
    eps = 1e-5
    for _ in range(6):
        v = np.zeros_like(X)
        for _ in range(3):
            cx, cy = rng.uniform(2.0, 22.0), rng.uniform(2.0, 16.0)
            v += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(2.0, 8.0))
        v *= 1e-4
        fdb = (_oracle_loss_state(sb, sb.w0 + eps * v, gauges, obs)
               - _oracle_loss_state(sb, sb.w0 - eps * v, gauges, obs)) / (2 * eps)
        fdn = (_oracle_loss_state(sn, sn.w0 + eps * v, gauges, obs)
               - _oracle_loss_state(sn, sn.w0 - eps * v, gauges, obs)) / (2 * eps)
        adb, adn = float(np.sum(gb * v)), float(np.sum(gn * v))
        assert abs(adb - fdb) <= 1e-3 * abs(fdb)
        assert abs((adb - adn) - (fdb - fdn)) <= 1e-2 * abs(fdb - fdn) + 1e-6 * abs(fdb)


@pytest.mark.parametrize("model", [0, 1], ids=["bsnq", "nlsw"])
def test_adjoint_corrector_matches_oracle_away_from_kinks(model):
    """One AM4 corrector iteration (K = 1): the reverse runs the corrector
    stage (its base Y, its right side at the predicted state, the sine
    ghosts at t^{n+1}) and then the predictor; a sine maker on the west."""
    from paper_1611_05984_gb300 import scenarios as sc
    s, gauges, X, Y = _tilted_bsnq(model, nsteps=10, K=1)
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.002, 4.0, 0.2, 0.3),))
    rng = np.random.default_rng(8)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, grad, _ = _gpu_gradient(s, gauges, obs, ckpt=3)
    assert abs(loss - _oracle_loss_state(s, s.w0, gauges, obs)) <= 1e-9 * loss
    eps = 1e-5
    for _ in range(5):
        v = np.zeros_like(X)
        for _ in range(3):
            cx, cy = rng.uniform(2.0, 22.0), rng.uniform(2.0, 16.0)
            v += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(2.0, 8.0))
        v *= 1e-4
        fd = (_oracle_loss_state(s, s.w0 + eps * v, gauges, obs)
              - _oracle_loss_state(s, s.w0 - eps * v, gauges, obs)) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-3 * abs(fd), (ad, fd)


def _oracle_loss_bed(s, z, gauges, obs):
    import dataclasses
    o = oracle_from(dataclasses.replace(s, z=z))
    _, P, Q = s.initial_state()
    o.set_state(s.w0, P, Q)
    o.set_gauges(gauges, 1, s.steps)
    o.step(s.steps)
    return 0.5 * float(np.sum((o.read_gauges(s.steps) - obs) ** 2))


def _tilted_bed(model, K, friction, nsteps=10):
    """The kink-free tilted state over a sloping, undulating bed (depth 0.35
    to 0.6 m, wet everywhere), sponge on the east, walls elsewhere."""
    s, gauges, X, Y = _tilted_bsnq(model, nsteps=nsteps, K=K)
    s.friction = friction
    xs, ys = X / (s.nx * s.dx), Y / (s.ny * s.dy)
    s.z = -0.5 + 0.08 * xs + 0.04 * ys ** 2 + 0.01 * np.sin(2 * math.pi * X / 6.0) * np.cos(2 * math.pi * Y / 9.0)
    return s, gauges, X, Y


@pytest.mark.parametrize("model,K,friction,sine", [(0, 0, 2, False), (0, 1, 1, False), (1, 1, 2, False),
                                                   (0, 1, 1, True), (1, 0, 2, True)],
                         ids=["bsnq-K0-manning", "bsnq-K1-quadratic", "nlsw-K1-manning",
                              "bsnq-K1-sine", "nlsw-K0-sine"])
def test_bed_gradient_matches_oracle_away_from_kinks(model, K, friction, sine):
    """dL/dz: the face beds of the reconstruction and the flux, the bed slope,
    friction, the dispersive and mixed terms' depth and the line systems'
    rows (Eq. 23), through the corners to the cell-centre bed; with a sine
    maker on the west also its ghost values, which follow the adjacent depth
    through the Eckart wave number (Eq. 25-29), in the fluxes, the dispersive
    terms and the line solves' boundary rows."""
    from paper_1611_05984_gb300 import scenarios as sc
    s, gauges, X, Y = _tilted_bed(model, K, friction)
    if sine:
        s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.002, 4.0, 0.2, 0.3), (0.001, 2.5, -0.3, 1.1)))
    rng = np.random.default_rng(21 + model + 2 * K)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, _, _, gz = _gpu_gradient(s, gauges, obs, ckpt=3, bed=True)
    assert abs(loss - _oracle_loss_bed(s, s.z, gauges, obs)) <= 1e-9 * loss
    # bed perturbations of 1e-7 m: the loss's rounding over the run (about
    # 1e-15 L) stays 4 orders below the difference
    eps = 1e-5
    errs = []
    for _ in range(5):
        v = np.zeros_like(X)
        for _ in range(3):
            cx, cy = rng.uniform(2.0, 22.0), rng.uniform(2.0, 16.0)
            v += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(2.0, 8.0))
        v *= 1e-2
        fd = (_oracle_loss_bed(s, s.z + eps * v, gauges, obs) - _oracle_loss_bed(s, s.z - eps * v, gauges, obs)) / (2 * eps)
        ad = float(np.sum(gz * v))
        errs.append(abs(ad - fd) / abs(fd))
    assert max(errs) <= 1e-3, errs


def test_bed_gradient_vertical_shift_identity_with_dry_land():
    """Shallow water (K = 1, Manning friction, walls, a beach with dry land):
    moving the given w0 and z up by c moves eta by c at every gauge and
    changes nothing else.  On dry cells w0 is the cell bed (the clamp), a
    path dL/dz already holds, so sum(dL/dw0 over wet cells) + sum(dL/dz) =
    sum over steps and gauges of (eta - obs)."""
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx = 48, 32, 0.5
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    z = np.maximum(-0.5, (X - 17.0) * 0.1)
    dt = 0.1 * dx / math.sqrt(9.81 * 0.5)
    s = sc.flat_basin(nx, ny, dx, 0.5, dt, model=1, K=1, friction=2, fcoef=0.02, eps=1e-8)
    s.z = z
    s.w0 = np.maximum(z, 0.05 * np.exp(-((X - 9.0) ** 2 + (Y - 8.0) ** 2) / 6.0))
    s.steps = 30
    rng = np.random.default_rng(13)
    gauges = [(int(rng.integers(4, 30)), int(rng.integers(3, ny - 3))) for _ in range(5)]
    obs = 0.005 * rng.standard_normal((s.steps, len(gauges)))
    loss, eta, gw, g, gz = _gpu_gradient(s, gauges, obs, ckpt=4, bed=True)
    bed = g.field("Bbar").double().cpu().numpy()
    wet = s.w0 > bed
    assert np.any(~wet) and np.any(gw[~wet] != 0.0)   # the shoreline's dry cells do matter
    want = float(np.sum(eta - obs))
    assert abs(float(np.sum(gw[wet]) + np.sum(gz)) - want) <= 1e-9 * np.sum(np.abs(eta - obs))
    # and the bed's gradient is not the trivial one: dry land follows the bed
    # (the clamp), the wet bed carries the rest
    land = z > 0.5
    assert np.all(gz[land] == 0.0) and np.linalg.norm(gz) > 0


def test_shift_identity_on_a_grid_of_16_row_tiles():
    """The same identity on a 1024 x 512 grid, large enough that the
    Jacobian pass takes its 32 x 16 tiles (the smaller grids above take
    32 x 8): a gentle beach with dry land, humps across the water and 40
    gauges spread over it, so that interior and boundary tiles of both
    kinds carry adjoints."""
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx = 1024, 512, 0.5
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    z = -0.5 + 1.5 * np.maximum(0.0, (X - 300.0) / 150.0)
    dt = 0.1 * dx / math.sqrt(9.81 * 0.5)
    s = sc.flat_basin(nx, ny, dx, 0.5, dt, model=1, K=1, friction=2, fcoef=0.02, eps=1e-8)
    s.z = z
    rng = np.random.default_rng(21)
    hump = np.zeros_like(X)
    for _ in range(12):
        x0, y0 = rng.uniform(5.0, 345.0), rng.uniform(5.0, 250.0)
        hump += 0.05 * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / 6.0)
    s.w0 = np.maximum(z, hump)
    s.steps = 30
    gauges = [(int(rng.integers(2, 700)), int(rng.integers(2, ny - 2))) for _ in range(40)]
    obs = 0.005 * rng.standard_normal((s.steps, len(gauges)))
    loss, eta, gw, g, gz = _gpu_gradient(s, gauges, obs, ckpt=0, bed=True)
    bed = g.field("Bbar").double().cpu().numpy()
    wet = s.w0 > bed
    want = float(np.sum(eta - obs))
    assert abs(float(np.sum(gw[wet]) + np.sum(gz)) - want) <= 1e-9 * np.sum(np.abs(eta - obs))
    assert np.count_nonzero(gw) > 40 * 100 and np.all(np.isfinite(gz))


def test_caller_scratch():
    """A caller-owned scratch tensor gives the gradients of an allocated
    one; a scratch below adjoint_scratch_bytes is refused before any work."""
    from paper_1611_05984_gb300 import celeris
    s, gauges = _scenario(nsteps=12)
    obs = torch.zeros((s.steps, len(gauges)), dtype=torch.float64)
    g1 = celeris.from_scenario(s, dtype=torch.float64)
    need = celeris.adjoint_scratch_bytes(g1, s.steps, len(gauges), 4, bed=True)
    scratch = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
    _, _, a_w, a_z = celeris.gauge_misfit_gradient(g1, s.steps, gauges, obs, 4, bed=True, scratch=scratch)
    g2 = celeris.from_scenario(s, dtype=torch.float64)
    _, _, b_w, b_z = celeris.gauge_misfit_gradient(g2, s.steps, gauges, obs, 4, bed=True)
    assert torch.linalg.norm(a_w - b_w) <= 1e-12 * torch.linalg.norm(b_w)
    assert torch.linalg.norm(a_z - b_z) <= 1e-12 * torch.linalg.norm(b_z)
    g3 = celeris.from_scenario(s, dtype=torch.float64)
    with pytest.raises(ValueError):
        celeris.gauge_misfit_gradient(g3, s.steps, gauges, obs, 4, bed=True,
                                      scratch=torch.empty(need - 1, dtype=torch.uint8, device="cuda"))


def test_adjoint_corrector_beach_with_dry_land():
    """K = 1 Boussinesq on a beach with dry land (dx = 0.5 m, depth/dx <=
    1): loss and records equal the oracle's, checkpoint spacing changes
    nothing, land far from the water gets zero gradient."""
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx = 48, 32, 0.5
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    z = np.maximum(-0.5, (X - 17.0) * 0.1)
    dt = 0.1 * dx / math.sqrt(9.81 * 0.5)
    s = sc.flat_basin(nx, ny, dx, 0.5, dt, model=0, K=1, friction=2, fcoef=0.02, eps=1e-8)
    s.z = z
    s.sides[sc.S] = sc.Side(sc.SPONGE, 5)
    s.w0 = np.maximum(z, 0.05 * np.exp(-((X - 9.0) ** 2 + (Y - 8.0) ** 2) / 6.0))
    s.steps = 30
    rng = np.random.default_rng(12)
    gauges = [(int(rng.integers(4, 30)), int(rng.integers(3, ny - 3))) for _ in range(5)]
    obs = 0.005 * rng.standard_normal((s.steps, len(gauges)))
    loss, eta, g4, g, z4 = _gpu_gradient(s, gauges, obs, ckpt=4, bed=True)
    lo, eta_o = _oracle_loss(s, s.w0, gauges, obs)
    assert abs(loss - lo) <= 1e-9 * abs(lo)
    np.testing.assert_allclose(eta, eta_o, rtol=0, atol=1e-11)
    _, _, g30, _, z30 = _gpu_gradient(s, gauges, obs, ckpt=30, bed=True)
    assert np.linalg.norm(g4 - g30) <= 1e-10 * np.linalg.norm(g30)
    assert np.linalg.norm(z4 - z30) <= 1e-10 * np.linalg.norm(z30)
    _, _, g0, _, z0 = _gpu_gradient(s, gauges, obs, ckpt=0, bed=True)   # every step kept
    assert np.linalg.norm(g0 - g30) <= 1e-10 * np.linalg.norm(g30)
    assert np.linalg.norm(z0 - z30) <= 1e-10 * np.linalg.norm(z30)
    land = z > 0.5
    assert np.any(land) and np.all(g4[land] == 0.0) and np.all(z4[land] == 0.0)
    assert np.linalg.norm(g4) > 0 and np.all(np.isfinite(z4)) and np.linalg.norm(z4) > 0


def _face_inputs(n, seed):
    """Seeded faces mixing deep, thin (h^4 below eps), dry and steep cells
    over sloping face beds, with their flux adjoints; columns as in
    cel_adjoint_face_selfcheck.  Also returns how often the reconstruction's
    positivity fix and the dry (zero wave speed) face occur."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 22))
    b0 = rng.uniform(-1.0, 0.2, n)
    sl = rng.normal(0.0, 0.05, n)
    Bface = b0[:, None] + sl[:, None] * np.array([-1.0, 0.0, 1.0]) + rng.normal(0.0, 0.01, (n, 3))
    bcell = b0[:, None] + sl[:, None] * np.array([-1.5, -0.5, 0.5, 1.5])
    kind = rng.integers(0, 5, (n, 4))
    h = np.where(kind == 0, rng.uniform(0.1, 1.0, (n, 4)),
                 np.where(kind == 1, 10.0 ** rng.uniform(-4, -2, (n, 4)),
                          np.where(kind == 2, 0.0, rng.uniform(0.0, 0.05, (n, 4)))))
    steep = kind == 4                                   # a jump across the cell
    w = bcell + h + np.where(steep, rng.normal(0.0, 0.3, (n, 4)), 0.0)
    w = np.maximum(w, bcell)
    wet = w > bcell
    x[:, 0:4] = w
    x[:, 4:8] = np.where(wet, rng.normal(0.0, 0.3, (n, 4)) * (w - bcell + 0.01), 0.0)
    x[:, 8:12] = np.where(wet, rng.normal(0.0, 0.3, (n, 4)) * (w - bcell + 0.01), 0.0)
    x[:, 12:15] = Bface
    x[:, 15:18] = rng.normal(0.0, 1.0, (n, 3))
    x[:, 18] = rng.uniform(1.0, 2.0, n)
    x[:, 19] = 9.81
    x[:, 20] = np.where(rng.random(n) < 0.5, 1e-8, 1e-12)
    x[:, 21] = rng.integers(0, 2, n)

    def mm(th, a0, a1, a2):
        a, b, c = th * (a1 - a0), 0.5 * (a2 - a0), th * (a2 - a1)
        lo, hi = np.minimum(a, np.minimum(b, c)), np.maximum(a, np.maximum(b, c))
        return np.where(lo > 0, lo, np.where(hi < 0, hi, 0.0))
    th = x[:, 18]
    sL, sR = mm(th, w[:, 0], w[:, 1], w[:, 2]), mm(th, w[:, 1], w[:, 2], w[:, 3])
    fixes = int(np.sum(w[:, 1] + 0.5 * sL < Bface[:, 1]) + np.sum(w[:, 1] - 0.5 * sL < Bface[:, 0])
                + np.sum(w[:, 2] + 0.5 * sR < Bface[:, 2]) + np.sum(w[:, 2] - 0.5 * sR < Bface[:, 1]))
    dry = int(np.sum((w[:, 1] <= Bface[:, 1]) & (w[:, 2] <= Bface[:, 1])))
    return x, fixes, dry


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_face_flux_vjp_by_hand_matches_dual_numbers(prec):
    """The reverse sweep's face-flux VJP is written by hand (one forward
    pass keeping its branches, then the adjoints back); here it is checked
    against the dual-number VJP of the forward's own flux code on faces that
    take every branch: the minmod's three slopes and zero, the positivity
    fix on either face of either cell, thin films below the
    desingularisation threshold, one- and two-sided dry faces."""
    from paper_1611_05984_gb300 import celeris
    x, fixes, dry = _face_inputs(20000, 17)
    assert fixes > 500 and dry > 200
    dtype = torch.float64 if prec == "f64" else torch.float32
    dual, hand = celeris.face_vjp_selfcheck(torch.as_tensor(x, dtype=dtype, device="cuda"))
    dual, hand = dual.double().cpu().numpy(), hand.double().cpu().numpy()
    assert np.count_nonzero(dual) > 0.3 * dual.size    # about 39 %: an outer cell counts only on some branches
    scale = np.maximum(np.max(np.abs(dual), axis=1, keepdims=True), 1e-30)
    err = np.max(np.abs(hand - dual) / scale, axis=1)
    if prec == "f64":
        assert np.max(err) <= 1e-10
    else:   # FP32: the two roundings may pick different sides of a near-tie in a few faces
        assert np.quantile(err, 0.999) <= 1e-3 and np.median(err) <= 1e-5


def test_gradients_on_32_random_directions():
    """Both gradients against FP64 central differences of the oracle along
    32 seeded random directions (16 in w0, 16 in z), each a random field
    smoothed over a few cells, on the kink-free Boussinesq state over the
    undulating bed with one AM4 corrector iteration: every one within 1e-3
    relative."""
    from scipy.ndimage import uniform_filter
    s, gauges, X, Y = _tilted_bed(0, 1, 2)
    rng = np.random.default_rng(32)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, gw, _, gz = _gpu_gradient(s, gauges, obs, ckpt=4, bed=True)
    assert abs(loss - _oracle_loss_bed(s, s.z, gauges, obs)) <= 1e-9 * loss
    eps = 1e-5
    errs = []
    for k in range(32):
        v = uniform_filter(rng.standard_normal(X.shape), size=5, mode="nearest")
        if k < 16:
            v *= 1e-4 / np.max(np.abs(v))
            fd = (_oracle_loss_state(s, s.w0 + eps * v, gauges, obs)
                  - _oracle_loss_state(s, s.w0 - eps * v, gauges, obs)) / (2 * eps)
            ad = float(np.sum(gw * v))
        else:
            v *= 1e-2 / np.max(np.abs(v))
            fd = (_oracle_loss_bed(s, s.z + eps * v, gauges, obs)
                  - _oracle_loss_bed(s, s.z - eps * v, gauges, obs)) / (2 * eps)
            ad = float(np.sum(gz * v))
        errs.append(abs(ad - fd) / abs(fd))
    assert max(errs) <= 1e-3, errs


@pytest.mark.parametrize("model", [0, 1], ids=["bsnq", "nlsw"])
def test_bed_gradient_through_the_sine_makers_ghosts(model):
    """The sine maker's ghost values (Eq. 25-28) follow the depth of the
    cell beside them: the wave number by Eckart (Eq. 29) and the celerity
    w / k.  A 3 cm + 2 cm maker, gauges in the first four columns and bed
    directions concentrated on the west columns make that path about 2 % of
    <dL/dz, v> (the celerity's depth derivative times the ghost discharge
    against the flux's own bed terms), so leaving it out would fail the 1e-3
    bound; a short run keeps the state off the limiter's kinks."""
    from paper_1611_05984_gb300 import scenarios as sc
    s, _, X, Y = _tilted_bed(model, 1, 1, nsteps=6)
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.03, 4.0, 0.2, 0.3), (0.02, 2.5, -0.3, 1.1)))
    gauges = [(i, j) for i in range(4) for j in (6, 13, 20, 27)]
    rng = np.random.default_rng(61 + model)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, _, _, gz = _gpu_gradient(s, gauges, obs, ckpt=2, bed=True)
    assert abs(loss - _oracle_loss_bed(s, s.z, gauges, obs)) <= 1e-9 * loss
    eps = 1e-5
    errs = []
    for _ in range(6):
        v = np.exp(-(X ** 2) / 1.0) * (1.0 + 0.5 * np.sin(2 * math.pi * Y / rng.uniform(4.0, 12.0) + rng.uniform(0, 6)))
        v *= 1e-2 * rng.choice([-1.0, 1.0])
        fd = (_oracle_loss_bed(s, s.z + eps * v, gauges, obs) - _oracle_loss_bed(s, s.z - eps * v, gauges, obs)) / (2 * eps)
        ad = float(np.sum(gz * v))
        errs.append(abs(ad - fd) / abs(fd))
    assert max(errs) <= 1e-3, errs


@pytest.mark.parametrize("model", [0, 1], ids=["bsnq", "nlsw"])
def test_gradients_with_two_corrector_iterations(model):
    """K = 2: every step reverses two AM4 stages (each with its own masks,
    solves, base and right side at the iterate before it) before the
    predictor; both gradients against oracle central differences."""
    from paper_1611_05984_gb300 import scenarios as sc
    s, gauges, X, Y = _tilted_bed(model, 2, 1, nsteps=8)
    s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.002, 4.0, 0.2, 0.3),))
    rng = np.random.default_rng(71 + model)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, gw, _, gz = _gpu_gradient(s, gauges, obs, ckpt=3, bed=True)
    assert abs(loss - _oracle_loss_bed(s, s.z, gauges, obs)) <= 1e-9 * loss
    eps = 1e-5
    errs = []
    for k in range(6):
        v = np.zeros_like(X)
        for _ in range(3):
            cx, cy = rng.uniform(2.0, 22.0), rng.uniform(2.0, 16.0)
            v += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(2.0, 8.0))
        if k < 3:
            v *= 1e-4
            fd = (_oracle_loss_state(s, s.w0 + eps * v, gauges, obs)
                  - _oracle_loss_state(s, s.w0 - eps * v, gauges, obs)) / (2 * eps)
            ad = float(np.sum(gw * v))
        else:
            v *= 1e-2
            fd = (_oracle_loss_bed(s, s.z + eps * v, gauges, obs)
                  - _oracle_loss_bed(s, s.z - eps * v, gauges, obs)) / (2 * eps)
            ad = float(np.sum(gz * v))
        errs.append(abs(ad - fd) / abs(fd))
    assert max(errs) <= 1e-3, errs


def _tlm_dl(s, gauges, obs, vz, vw):
    """dL along (vz, vw) from the tangent-linear oracle: L = 1/2 sum (eta -
    obs)^2 gives dL = sum (eta - obs) d eta."""
    from tests.helpers import tangent_run
    eta, deta = tangent_run(s, gauges, vz, vw)
    return float(np.sum((eta - obs) * deta))


@pytest.mark.parametrize("model,K,sine", [(0, 1, True), (1, 0, True), (0, 2, False)],
                         ids=["bsnq-K1-sine", "nlsw-K0-sine", "bsnq-K2"])
def test_adjoint_against_tangent_linear_oracle(model, K, sine):
    """The FP64 tangent-linear reference: the oracle's own arithmetic on dual
    numbers gives dL(x; v) exactly, with no step size; the adjoint's
    <dL/dw0, vw> + <dL/dz, vz> must equal it along joint random directions
    in the initial state and the bed, on the kink-free state."""
    from tests.helpers import tilted_bed_scenario
    s, gauges, X, Y = tilted_bed_scenario(model=model, K=K, friction=2, nsteps=10, sine=sine)
    rng = np.random.default_rng(90 + model + 3 * K)
    obs = 0.01 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, gw, _, gz = _gpu_gradient(s, gauges, obs, ckpt=3, bed=True)
    errs = []
    for _ in range(8):
        vw = rng.standard_normal(X.shape)
        vz = rng.standard_normal(X.shape)
        ref = _tlm_dl(s, gauges, obs, vz, vw)
        ad = float(np.sum(gw * vw) + np.sum(gz * vz))
        errs.append(abs(ad - ref) / abs(ref))
    # measured 1.4e-14 at most: the adjoint is the exact transpose of the
    # tangent, to rounding
    assert max(errs) <= 1e-12, errs


def test_adjoint_against_tangent_linear_oracle_on_a_beach():
    """A K = 1 beach with dry land and a moving shoreline: the state crosses
    the limiter's and the wet-dry branches.  Both codes take the same branch
    everywhere but at exact ties, where each takes one of the two one-sided
    derivatives: a dry cell whose update lands exactly on the bed counts as
    clamped in the adjoint (its adjoint goes to the bed) and as not clamped
    in the oracle (w < Bbar is false).  Measured: 6.8e-4 of the directional
    derivative at most, inside the 1e-3 bar."""
    from paper_1611_05984_gb300 import scenarios as sc
    nx, ny, dx = 48, 32, 0.5
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    z = np.maximum(-0.5, (X - 17.0) * 0.1)
    dt = 0.1 * dx / math.sqrt(9.81 * 0.5)
    s = sc.flat_basin(nx, ny, dx, 0.5, dt, model=0, K=1, friction=2, fcoef=0.02, eps=1e-8)
    s.z = z
    s.sides[sc.S] = sc.Side(sc.SPONGE, 5)
    s.w0 = np.maximum(z, 0.05 * np.exp(-((X - 9.0) ** 2 + (Y - 8.0) ** 2) / 6.0))
    s.steps = 30
    rng = np.random.default_rng(12)
    gauges = [(int(rng.integers(4, 30)), int(rng.integers(3, ny - 3))) for _ in range(5)]
    obs = 0.005 * rng.standard_normal((s.steps, len(gauges)))
    loss, _, gw, g, gz = _gpu_gradient(s, gauges, obs, ckpt=4, bed=True)
    bed = g.field("Bbar").double().cpu().numpy()
    wet = s.w0 > bed
    errs = []
    for _ in range(8):
        vw = rng.standard_normal(X.shape) * wet   # the clamp holds w0 at the bed on dry cells
        vz = rng.standard_normal(X.shape)
        ref = _tlm_dl(s, gauges, obs, vz, vw)
        ad = float(np.sum(gw * vw) + np.sum(gz * vz))
        errs.append(abs(ad - ref) / abs(ref))
    assert max(errs) <= 1e-3, errs


@pytest.mark.parametrize("steps,ckpt,bound", [(40, 10, 1e-12), (2000, 100, 1e-3)], ids=["40-steps", "2000-steps"])
def test_adjoint_against_tangent_linear_oracle_on_the_hump_beach(steps, ckpt, bound):
    """The adjoint's own configuration (the 512 x 512 hump beach, Boussinesq,
    K = 1, 16 gauges, observations from the perturbed-hump, perturbed-bed
    target run), over its first 40 steps (checkpoints every 10) and its full
    2000 (every 100): both gradients against the tangent-linear oracle along
    smooth random directions in the initial state and the bed."""
    from paper_1611_05984_gb300 import scenarios as sc
    from tests.helpers import tangent_run
    s, gauges = sc.hump_beach(n=512, steps=steps)
    t = oracle_from(sc.hump_beach_target(s))
    t.set_gauges(gauges, 1, s.steps)
    t.step(s.steps)
    obs = t.read_gauges(s.steps)
    loss, eta, gw, g, gz = _gpu_gradient(s, gauges, obs, ckpt=ckpt, bed=True)
    bed = g.field("Bbar").double().cpu().numpy()
    wet = s.w0 > bed
    X, Y = np.meshgrid(np.arange(s.nx) + 0.5, np.arange(s.ny) + 0.5)
    rng = np.random.default_rng(512)
    errs = []
    for _ in range(3):
        vw = np.zeros_like(X)
        vz = np.zeros_like(X)
        for _ in range(4):
            cx, cy, r = rng.uniform(100, 380), rng.uniform(60, 450), rng.uniform(15, 50)
            vw += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / r ** 2)
            vz += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / r ** 2)
        vw *= wet
        e, de = tangent_run(s, gauges, vz, vw)
        ref = float(np.sum((e - obs) * de))
        ad = float(np.sum(gw * vw) + np.sum(gz * vz))
        errs.append(abs(ad - ref) / abs(ref))
    print("tlm hump", steps, errs)
    assert max(errs) <= bound, errs


@pytest.mark.parametrize("steps", [500, 2000])
def test_fp32_gradients_on_the_hump_beach(steps):
    """The benchmark's precision: on the 512 x 512 hump beach (checkpoints
    every 100) the FP32 adjoint's gradients against the FP64 adjoint's
    (which equals the tangent-linear reference within 5e-5 at 2000 steps).
    Before the wave reaches the beach (500 steps) both gradients agree
    within 5e-3.  After it runs up the beach (2000 steps) the moving
    shoreline's wet-dry and limiter branches differ between the two
    precisions' states, and dL/dw0 -- the adjoint after all 2000 reversed
    steps -- carries those differences (6 % measured); dL/dz, summed over the
    run, stays within 1e-3.  Directional errors are scaled by the directions'
    rms derivative (a single direction can nearly cancel).  The hump is
    clipped at 4 widths so that both precisions see the same exact rest far
    away (an unclipped Gaussian's 1e-44 tail exists in FP64 only)."""
    from paper_1611_05984_gb300 import scenarios as sc
    s, gauges = sc.hump_beach(n=512, steps=steps)
    X, Y = np.meshgrid(np.arange(s.nx) + 0.5, np.arange(s.ny) + 0.5)
    r2 = (X - 0.4 * s.nx) ** 2 + (Y - 0.5 * s.ny) ** 2
    s.w0 = np.where(r2 < (4 * 30.0) ** 2, s.w0, np.maximum(s.z, 0.0))
    t = oracle_from(sc.hump_beach_target(s))
    t.set_gauges(gauges, 1, s.steps)
    t.step(s.steps)
    obs = t.read_gauges(s.steps)
    _, _, w64, g, z64 = _gpu_gradient(s, gauges, obs, ckpt=100, bed=True)
    _, _, w32, _, z32 = _gpu_gradient(s, gauges, obs, prec="f32", ckpt=100, bed=True)
    bed = g.field("Bbar").double().cpu().numpy()
    wet = s.w0 > bed
    rng = np.random.default_rng(32)
    d32, d64 = [], []
    for _ in range(8):
        vw = np.zeros_like(X)
        vz = np.zeros_like(X)
        for _ in range(4):
            cx, cy, r = rng.uniform(100, 380), rng.uniform(60, 450), rng.uniform(15, 50)
            vw += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / r ** 2)
            vz += rng.standard_normal() * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / r ** 2)
        vw *= wet
        d64.append(float(np.sum(w64 * vw) + np.sum(z64 * vz)))
        d32.append(float(np.sum(w32 * vw) + np.sum(z32 * vz)))
    d32, d64 = np.array(d32), np.array(d64)
    dirs = np.max(np.abs(d32 - d64)) / np.sqrt(np.mean(d64 ** 2))
    fw = np.linalg.norm((w32 - w64)[wet]) / np.linalg.norm(w64[wet])
    fz = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
    assert fz <= 1e-3, fz
    if steps == 500:
        assert fw <= 5e-3 and dirs <= 5e-3, (fw, dirs)
    else:
        assert fw <= 0.1 and dirs <= 0.05, (fw, dirs)


@pytest.mark.parametrize("model,K", [(0, 1), (1, 2)], ids=["bsnq-K1", "nlsw-K2"])
def test_adjoint_reads_nothing_unwritten(model, K):
    """The solver's workspace and the adjoint's scratch filled with 0xFF
    bytes (NaN in every real field) beforehand: the loss, the records and
    both gradients equal those of fresh allocations (to the atomics'
    summation order), with a sine maker, so the reverse's own ghost table,
    the ghost adjoints, both segment slots and the captured right sides are
    all exercised."""
    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc
    from tests.helpers import tilted_bed_scenario
    s, gauges, _, _ = tilted_bed_scenario(model=model, K=K, friction=2, nsteps=12, sine=True)
    rng = np.random.default_rng(3)
    obs = torch.as_tensor(0.01 * rng.standard_normal((s.steps, len(gauges))), dtype=torch.float64)
    out = []
    for poison in (False, True):
        g = celeris.from_scenario(s, dtype=torch.float64, poison=poison)
        out.append(celeris.gauge_misfit_gradient(g, s.steps, gauges, obs, 3, bed=True, poison=poison))
    (l0, e0, w0, z0), (l1, e1, w1, z1) = out
    assert l1 == pytest.approx(l0, rel=1e-14)
    assert torch.equal(e0, e1)
    for a, b in ((w0, w1), (z0, z1)):
        assert torch.isfinite(b).all()
        assert float(torch.linalg.norm(b - a)) <= 1e-12 * float(torch.linalg.norm(a))
