"""The fixed-scratch entry point, cel_advance_noalloc, against the workspace path.

cel_advance_noalloc is for callers that cannot allocate device memory: code
living inside a host application that owns the GPU's memory pool, real-time
loops that must not call cudaMalloc/cudaFree after start-up (both can
synchronise the device), and thin bindings that can pass a stream and a few
existing buffers but cannot allocate.  It keeps its scratch in one array the
library defines in device memory, shared by all calls.

The test calls it twice in a row through the C ABI, each time from a
different state, and compares each result with what cel_create +
cel_set_boundary + cel_set_state + cel_step + cel_get_state give for the same
input.  Both paths launch the same kernels on the same inputs, so the results
must be equal bit for bit (which is within any tolerance of the other GPU
tests); a scratch value left over from the first call would show up in the
second.  A third case starts at first_step = N, where the sine maker's phase
depends on the start time.  This file is named so that pytest collects it
last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-10, torch.float32: 1e-4}


def _rel(a, b):
    a, b = a.double(), b.double()
    den = torch.linalg.norm(b).item()
    return torch.linalg.norm(a - b).item() / (den if den > 0 else 1.0)


def _bcs(scenario, celeris):
    arr = (celeris.CelBC * 4)()
    for side in range(4):
        sd = scenario.sides.get(side)
        if sd is not None:
            arr[side] = celeris.make_bc(sd.type, sd.width, sd.comps)
    return arr


def _noalloc(celeris, s, dtype, state, nsteps, first_step=0):
    L = celeris.load()
    es = 4 if dtype == torch.float32 else 8
    grid = celeris.CelGrid(s.nx, s.ny, s.dx, s.dy, es)
    params = celeris.CelParams(s.model, s.g, s.Bd, s.theta, s.eps, s.dt, s.K, s.ws, s.friction, s.fcoef)
    z = torch.as_tensor(s.z, dtype=dtype, device="cuda").contiguous()
    w, P, Q = (t.to(device="cuda", dtype=dtype).contiguous() for t in state)
    out = [torch.empty_like(w) for _ in range(3)]
    msg = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    st = L.cel_advance_noalloc(ctypes.byref(grid), ctypes.byref(params), _bcs(s, celeris), z.data_ptr(),
                               w.data_ptr(), P.data_ptr(), Q.data_ptr(), out[0].data_ptr(),
                               out[1].data_ptr(), out[2].data_ptr(), nsteps, first_step, stream.cuda_stream,
                               msg, len(msg))
    assert st == 0, msg.value.decode()
    stream.synchronize()
    return out


def _workspace_path(celeris, s, dtype, state, nsteps, first_step=0):
    g = celeris.Solver(s.z, s.dx, s.dy, s.dt, dtype=dtype, model=s.model, g=s.g, Bd=s.Bd, theta=s.theta,
                       eps=s.eps, K=s.K, ws=s.ws, friction=s.friction, fcoef=s.fcoef)
    for side, sd in s.sides.items():
        g.set_boundary(side, sd.type, sd.width, sd.comps)
    g.set_state(*state)
    if first_step:
        # run to step first_step, then restart the history from the given
        # state: set_state keeps the step count (the time), so the next steps
        # start at first_step * dt with Euler steps, as the entry point does
        g.step(first_step)
        assert g.time()[1] == first_step
        g.set_state(*state)
    g.step(nsteps)
    return list(g.state())


def _same(a, b, dtype):
    assert _rel(a, b) <= TOL[dtype]
    assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_noalloc_matches_workspace_path_on_two_calls(dtype):
    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc

    s = sc.beach(nx=200, ny=150, sponge=20)            # sine maker, sponges, K = 1
    rest = [torch.as_tensor(a, dtype=dtype) for a in s.initial_state()]
    first = _noalloc(celeris, s, dtype, rest, 120)
    ref1 = _workspace_path(celeris, s, dtype, rest, 120)
    for a, b in zip(first, ref1):
        _same(a, b, dtype)

    # second call in a row, from a different state (the first result with a
    # trough added), fewer steps
    w2, P2, Q2 = (t.clone() for t in first)
    w2[40:60, 30:50] -= 0.05
    second = _noalloc(celeris, s, dtype, [w2, P2, Q2], 80)
    ref2 = _workspace_path(celeris, s, dtype, [w2, P2, Q2], 80)
    for a, b in zip(second, ref2):
        _same(a, b, dtype)
    assert not torch.equal(second[0], first[0])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_noalloc_start_step_sets_the_sine_makers_phase(dtype):
    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc

    s = sc.beach(nx=160, ny=96, sponge=12)
    rest = [torch.as_tensor(a, dtype=dtype) for a in s.initial_state()]
    late = _noalloc(celeris, s, dtype, rest, 60, first_step=137)
    ref = _workspace_path(celeris, s, dtype, rest, 60, first_step=137)
    for a, b in zip(late, ref):
        _same(a, b, dtype)
    # the maker's phase moved with the start time: a run from step 0 differs
    early = _noalloc(celeris, s, dtype, rest, 60)
    assert not torch.equal(late[0], early[0])


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    from paper_1611_05984_gb300 import celeris
    L = celeris.load()
    grid = celeris.CelGrid(2048, 2048, 1.0, 1.0, 4)
    params = celeris.CelParams(0, 9.81, 1 / 15, 1.3, 1e-8, 0.01, 1, 0.0, 2, 0.015)
    msg = ctypes.create_string_buffer(256)
    buf = torch.zeros(16, device="cuda")
    p = buf.data_ptr()
    st = L.cel_advance_noalloc(ctypes.byref(grid), ctypes.byref(params), None, p, p, p, p, p, p, p, 1, 0,
                               None, msg, len(msg))
    assert st == 2                                     # CEL_ERR_WORKSPACE_TOO_SMALL
    assert b"fixed scratch holds" in msg.value
