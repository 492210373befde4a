"""FP64 CPU oracle of the Celeris extended-Boussinesq time step (arXiv 1611.05984).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
restatement of the paper's method that the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA
library (``paper_1611_05984_gb300``) and never imports it.

Parity-pin status of the oracle's parts (the tests under ``tests/`` that pin
each one are named in the test module docstrings):
  * reconstruction, flux, bed slope: lake at rest (well-balanced) -- pinned
  * flux form, walls, AB3: mass conservation with solid walls -- pinned
  * KP07 NLSW path + dry front: Ritter dam-break closed form -- pinned
  * dispersion + tridiagonal + F*: linear dispersion relation -- pinned
  * depth-gradient terms of Eq. 10-11 and Eq. 23: linear shoaling on a
    slope -- pinned; those of F*, G* (Eq. 12-13) and the cross terms of
    Eq. 10-11, which vanish in 1-D: isotropy over a round shoal (eta along
    the diagonals converges to eta along the axes) -- pinned.
  * mirror / transpose symmetry -- pinned
  * Thomas solver: dense solve -- pinned; Eckart, sponge, soliton -- pinned
  * friction + AB3 order: uniform-flow ODE -- pinned
  * Euler start-up, AB3 predictor and AM4 corrector iterations: each step's
    formula on the friction ODE, to rounding -- pinned
  * sine maker: the wave it sends into a sponged channel is progressive,
    P = c eta with the model's dispersion relation, amplitude a, and its
    steady phase converged in dt (the stages' ghost times) -- pinned
  * corner ghosts: beside a wall, exact embedding in a run twice as high
    -- pinned; where two sine makers meet, the plane wave both send is kept
    at the corner (phase steps and amplitude within a few per cent) --
    pinned.
  * run-up tracking: standing-mode maximum, dry threshold -- pinned
  * tangent-linear oracle (celeris_tlm.cpp: this source on dual numbers):
    values bit for bit the oracle's, tangents vs central differences,
    linearity -- pinned (tests/test_tlm_oracle.py).
  * render oracle (render_oracle.c, the headless renderer): Fresnel closed
    forms, colormap control points, flat lake / tilted plane / flat land by
    formula, grid lines, speed, mirror symmetry -- pinned
    (tests/test_render_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "celeris_oracle.c")
_HDR = os.path.join(_HERE, "celeris_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libceleris_oracle.so")
_lock = threading.Lock()
_lib = None

BSNQ, NLSW = 0, 1
FRIC_NONE, FRIC_QUAD, FRIC_MANNING = 0, 1, 2
SOLID, SPONGE, SINE = 0, 1, 2
W, E, S, N = 0, 1, 2, 3


class OrcParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("model", ctypes.c_int), ("g", ctypes.c_double),
                ("Bd", ctypes.c_double), ("theta", ctypes.c_double),
                ("eps", ctypes.c_double), ("dt", ctypes.c_double),
                ("K", ctypes.c_int), ("ws", ctypes.c_double),
                ("friction", ctypes.c_int), ("fcoef", ctypes.c_double)]


class OrcBC(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("width", ctypes.c_int),
                ("ncomp", ctypes.c_int),
                ("amp", ctypes.c_double * 8), ("period", ctypes.c_double * 8),
                ("dir", ctypes.c_double * 8), ("phase", ctypes.c_double * 8)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, FP64, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation test load a deliberately broken copy
            path = os.environ.get("ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_create.restype = p
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams), dp]
            L.orc_destroy.argtypes = [p]
            L.orc_set_boundary.argtypes = [p, i, ctypes.POINTER(OrcBC)]
            L.orc_set_state.argtypes = [p, dp, dp, dp]
            L.orc_add_solitary.argtypes = [p, d, d, d, d]
            L.orc_step.argtypes = [p, i]
            L.orc_get_state.argtypes = [p, dp, dp, dp]
            L.orc_get_field.argtypes = [p, i, dp]
            L.orc_get_time.argtypes = [p, dp, ctypes.POINTER(ctypes.c_longlong)]
            L.orc_mass.restype = d
            L.orc_mass.argtypes = [p]
            L.orc_clamp_mass.restype = d
            L.orc_clamp_mass.argtypes = [p]
            L.orc_set_gauges.argtypes = [p, ctypes.POINTER(ctypes.c_int), i, i, i]
            L.orc_read_gauges.argtypes = [p, dp, i, ctypes.POINTER(ctypes.c_int)]
            L.orc_runup_enable.argtypes = [p, d]
            L.orc_runup_read.argtypes = [p, dp]
            L.orc_num_threads.restype = i
            L.orc_minmod.restype = d
            L.orc_minmod.argtypes = [d, d, d, d]
            L.orc_eckart_k.restype = d
            L.orc_eckart_k.argtypes = [d, d, d]
            L.orc_sponge_gamma.restype = d
            L.orc_sponge_gamma.argtypes = [d, d]
            L.orc_thomas.argtypes = [i, dp, dp, dp, dp, dp]
            L.orc_central_upwind.argtypes = [d] * 9 + [dp]
            _lib = L
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def make_bc(type=SOLID, width=0, comps=()):
    """comps: iterable of (amp, period, dir_rad, phase_rad)."""
    bc = OrcBC()
    bc.type, bc.width, bc.ncomp = int(type), int(width), len(comps)
    for m, (a, T, th, ph) in enumerate(comps):
        bc.amp[m], bc.period[m], bc.dir[m], bc.phase[m] = a, T, th, ph
    return bc


class Oracle:
    """One oracle simulation.  Arguments mirror the paper's problem statement."""

    def __init__(self, z, dx, dy, dt, *, model=BSNQ, g=9.81, Bd=1.0 / 15.0,
                 theta=1.3, eps=5e-12, K=0, ws=0.0, friction=FRIC_NONE, fcoef=0.0):
        z = _f64(z)
        ny, nx = z.shape
        self.nx, self.ny = nx, ny
        self.p = OrcParams(nx, ny, dx, dy, model, g, Bd, theta, eps, dt, K, ws,
                           friction, fcoef)
        self._L = lib()
        self._h = self._L.orc_create(ctypes.byref(self.p), _dp(z))
        if not self._h:
            raise ValueError("orc_create rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    def set_boundary(self, side, type=SOLID, width=0, comps=()):
        bc = make_bc(type, width, comps)
        if self._L.orc_set_boundary(self._h, side, ctypes.byref(bc)) != 0:
            raise ValueError("bad boundary")

    def set_state(self, w, P, Q):
        sh = (self.ny, self.nx)
        w, P, Q = _f64(w, sh), _f64(P, sh), _f64(Q, sh)
        if self._L.orc_set_state(self._h, _dp(w), _dp(P), _dp(Q)) != 0:
            raise ValueError("bad state")

    def add_solitary(self, H, theta, x0, y0):
        if self._L.orc_add_solitary(self._h, H, theta, x0, y0) != 0:
            raise ValueError("solitary wave rejected (dry crest)")

    def step(self, n=1):
        if self._L.orc_step(self._h, int(n)) != 0:
            raise RuntimeError("orc_step failed")

    def state(self):
        sh = (self.ny, self.nx)
        w, P, Q = np.empty(sh), np.empty(sh), np.empty(sh)
        self._L.orc_get_state(self._h, _dp(w), _dp(P), _dp(Q))
        return w, P, Q

    def field(self, which):
        idx = {"Bbar": 0, "d": 1, "U": 2, "V": 3}[which]
        out = np.empty((self.ny, self.nx))
        self._L.orc_get_field(self._h, idx, _dp(out))
        return out

    def time(self):
        t = ctypes.c_double()
        s = ctypes.c_longlong()
        self._L.orc_get_time(self._h, ctypes.byref(t), ctypes.byref(s))
        return t.value, s.value

    def mass(self):
        return self._L.orc_mass(self._h)

    def clamp_mass(self):
        return self._L.orc_clamp_mass(self._h)

    def set_gauges(self, ij, log_every, capacity):
        ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
        ptr = ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if self._L.orc_set_gauges(self._h, ptr, len(ij), log_every, capacity) != 0:
            raise ValueError("bad gauges")
        self._ng = len(ij)

    def read_gauges(self, max_rec):
        out = np.zeros((max_rec, self._ng))
        n = ctypes.c_int()
        self._L.orc_read_gauges(self._h, _dp(out), max_rec, ctypes.byref(n))
        return out[: n.value]


    def runup_enable(self, delta):
        """Track the highest w seen where the depth exceeds delta (Sec. 4.1,
        4.3), starting from the present state."""
        if self._L.orc_runup_enable(self._h, float(delta)) != 0:
            raise ValueError("bad run-up threshold")

    def runup(self):
        """(ny, nx) highest w seen while wetter than the threshold; -inf where
        never."""
        out = np.empty((self.ny, self.nx))
        if self._L.orc_runup_read(self._h, _dp(out)) != 0:
            raise ValueError("run-up tracking is not enabled")
        return out


def minmod(theta, qm, q0, qp):
    return lib().orc_minmod(theta, qm, q0, qp)


def eckart_k(omega, d, g=9.81):
    return lib().orc_eckart_k(omega, d, g)


def sponge_gamma(D, Ls):
    return lib().orc_sponge_gamma(D, Ls)


def thomas(a, b, c, r):
    a, b, c, r = (_f64(v) for v in (a, b, c, r))
    x = np.empty_like(r)
    lib().orc_thomas(len(r), _dp(a), _dp(b), _dp(c), _dp(r), _dp(x))
    return x


def central_upwind(g, eps, wL, nL, tL, wR, nR, tR, Bf):
    H = np.zeros(3)
    lib().orc_central_upwind(g, eps, wL, nL, tL, wR, nR, tR, Bf, _dp(H))
    return H


def num_threads():
    return lib().orc_num_threads()


# ------------------------------------------------------------------ render
# CPU restatement of the headless renderer (render_oracle.c): a separate
# library, single precision, one rounded operation at a time.

_RSRC = os.path.join(_HERE, "render_oracle.c")
_RHDR = os.path.join(_HERE, "render_oracle.h")
_RLIB = os.path.join(_HERE, "_build", "librender_oracle.so")
_rlib = None

RENDER_MODES = {"eta": 0, "u": 1, "v": 2, "speed": 3, "fresnel": 4}


class RoParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("vmin", ctypes.c_float), ("vmax", ctypes.c_float),
                ("dry_h", ctypes.c_float), ("h_min", ctypes.c_float), ("zmin", ctypes.c_float),
                ("zmax", ctypes.c_float), ("grid", ctypes.c_float), ("exaggeration", ctypes.c_float),
                ("view", ctypes.c_float * 3), ("sun", ctypes.c_float * 3), ("absorb", ctypes.c_float)]


def build_render(force: bool = False) -> str:
    """Compile the render oracle (plain C99, single precision, no FMA contraction)."""
    os.makedirs(os.path.dirname(_RLIB), exist_ok=True)
    newest = max(os.path.getmtime(_RSRC), os.path.getmtime(_RHDR))
    if not force and os.path.exists(_RLIB) and os.path.getmtime(_RLIB) >= newest:
        return _RLIB
    tmp = _RLIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _RSRC, "-lm"],
                   check=True)
    os.replace(tmp, _RLIB)
    return _RLIB


def render_lib():
    global _rlib
    with _lock:
        if _rlib is None:
            L = ctypes.CDLL(os.environ.get("RENDER_ORACLE_LIB") or build_render())
            dp = ctypes.POINTER(ctypes.c_double)
            L.ro_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    dp, dp, dp, dp, ctypes.POINTER(RoParams), ctypes.c_void_p]
            L.ro_fresnel.restype = ctypes.c_float
            L.ro_fresnel.argtypes = [ctypes.c_float]
            L.ro_colormap.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
            _rlib = L
        return _rlib


def render_params(mode="eta", vmin=-1.0, vmax=1.0, dry_h=1e-3, h_min=1e-2, zmin=-1.0, zmax=1.0, grid=0.0,
                  exaggeration=1.0, view=(0.0, 0.0, -1.0), sun=(0.3, 0.4, 1.0), absorb=0.5) -> RoParams:
    return RoParams(RENDER_MODES[mode] if isinstance(mode, str) else int(mode), vmin, vmax, dry_h, h_min, zmin,
                    zmax, grid, exaggeration, (ctypes.c_float * 3)(*view), (ctypes.c_float * 3)(*sun), absorb)


def render(w, P, Q, Bbar, dx, dy, ws=0.0, params: RoParams = None) -> np.ndarray:
    """RGBA image (ny, nx, 4) uint8 of the state (row j = grid row j)."""
    w, P, Q, Bbar = (_f64(a) for a in (w, P, Q, Bbar))
    ny, nx = w.shape
    out = np.zeros((ny, nx, 4), np.uint8)
    p = params or render_params()
    render_lib().ro_render(nx, ny, dx, dy, ws, _dp(w), _dp(P), _dp(Q), _dp(Bbar), ctypes.byref(p),
                           out.ctypes.data_as(ctypes.c_void_p))
    return out


def fresnel(cos_i):
    return render_lib().ro_fresnel(cos_i)


def colormap(which, t):
    out = (ctypes.c_float * 3)()
    render_lib().ro_colormap(which, t, out)
    return np.array(out[:], np.float32)


# ------------------------------------------------- tangent-linear oracle
#
# celeris_tlm.cpp compiles celeris_oracle.c again with a forward-mode dual
# number as its arithmetic type: the tangent of every output along one
# direction (dz, dw, dP, dQ) of the inputs, the exact directional derivative
# of the oracle's own arithmetic and branches.  The discrete adjoint's
# gradients are checked against it: <dL/dx, v> must equal dL(x; v).

_TLM_SRC = os.path.join(_HERE, "celeris_tlm.cpp")
_TLM_LIB = os.path.join(_HERE, "_build", "libceleris_tlm.so")
_tlm = None


def build_tlm(force: bool = False) -> str:
    """Compile the tangent-linear oracle (g++, FP64, no FMA contraction, OpenMP over rows and lines as
    the oracle)."""
    os.makedirs(os.path.dirname(_TLM_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(_TLM_SRC))
    if not force and os.path.exists(_TLM_LIB) and os.path.getmtime(_TLM_LIB) >= newest:
        return _TLM_LIB
    tmp = _TLM_LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _TLM_SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _TLM_LIB)
    return _TLM_LIB


def tlm_lib():
    global _tlm
    with _lock:
        if _tlm is None:
            # TLM_ORACLE_LIB lets the mutation test load a deliberately broken copy
            L = ctypes.CDLL(os.environ.get("TLM_ORACLE_LIB") or build_tlm())
            i, p = ctypes.c_int, ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            L.tlm_create.restype = p
            L.tlm_create.argtypes = [ctypes.POINTER(OrcParams), dp, dp]
            L.tlm_destroy.argtypes = [p]
            L.tlm_set_boundary.argtypes = [p, i, ctypes.POINTER(OrcBC)]
            L.tlm_set_state.argtypes = [p, i, dp, dp, dp, dp, dp, dp]
            L.tlm_set_gauges.argtypes = [p, ctypes.POINTER(ctypes.c_int), i, i, i]
            L.tlm_step.argtypes = [p, i]
            L.tlm_read_gauges.argtypes = [p, dp, dp, i, i, ctypes.POINTER(ctypes.c_int)]
            _tlm = L
        return _tlm


class TangentOracle:
    """The oracle with a tangent: the bed z with its direction dz; then
    set_state(w, P, Q, dw, dP, dQ); gauges read as (eta, d eta)."""

    def __init__(self, z, dz, dx, dy, dt, *, model=BSNQ, g=9.81, Bd=1.0 / 15.0,
                 theta=1.3, eps=5e-12, K=0, ws=0.0, friction=FRIC_NONE, fcoef=0.0):
        z = _f64(z)
        ny, nx = z.shape
        dz = _f64(dz, (ny, nx))
        self.nx, self.ny, self.ng = nx, ny, 0
        self.p = OrcParams(nx, ny, dx, dy, model, g, Bd, theta, eps, dt, K, ws, friction, fcoef)
        self._L = tlm_lib()
        self._h = self._L.tlm_create(ctypes.byref(self.p), _dp(z), _dp(dz))
        if not self._h:
            raise ValueError("tlm_create rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.tlm_destroy(h)
            self._h = None

    def set_boundary(self, side, type=SOLID, width=0, comps=()):
        bc = make_bc(type, width, comps)
        if self._L.tlm_set_boundary(self._h, side, ctypes.byref(bc)) != 0:
            raise ValueError("bad boundary")

    def set_state(self, w, P, Q, dw, dP, dQ):
        sh = (self.ny, self.nx)
        a = [_f64(x, sh) for x in (w, dw, P, dP, Q, dQ)]
        if self._L.tlm_set_state(self._h, self.nx * self.ny, *[_dp(x) for x in a]) != 0:
            raise ValueError("bad state")

    def set_gauges(self, ij, log_every, capacity):
        ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
        self.ng = len(ij)
        if self._L.tlm_set_gauges(self._h, ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(ij),
                                  int(log_every), int(capacity)) != 0:
            raise ValueError("bad gauges")

    def step(self, n=1):
        if self._L.tlm_step(self._h, int(n)) != 0:
            raise RuntimeError("tlm_step failed")

    def read_gauges(self, max_rec):
        eta, deta = np.zeros((max_rec, self.ng)), np.zeros((max_rec, self.ng))
        n = ctypes.c_int()
        if self._L.tlm_read_gauges(self._h, _dp(eta), _dp(deta), int(max_rec), self.ng, ctypes.byref(n)) != 0:
            raise RuntimeError("tlm_read_gauges failed")
        return eta[: n.value], deta[: n.value]
