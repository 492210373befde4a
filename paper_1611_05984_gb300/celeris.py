"""Python binding of the Celeris GB300 step library (ctypes over the C ABI).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libceleris_gb.so``.  PyTorch supplies the device memory (the workspace,
gauge ring and checkpoint buffers are torch tensors the binding keeps alive)
and the CUDA stream (``torch.cuda.current_stream()`` by default).  There is no
CPU fallback: constructing a Solver without a CUDA device or without the
compiled library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

CEL_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "workspace too small", 3: "CUDA error",
          4: "non-finite value", 5: "timeout", 6: "not implemented"}
BSNQ, NLSW = 0, 1
FRIC_NONE, FRIC_QUADRATIC, FRIC_MANNING = 0, 1, 2
SOLID, SPONGE, SINE = 0, 1, 2
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
FIELDS = {"Bbar": 0, "d": 1, "U": 2, "V": 3}

EXPORTS = ["cel_workspace_bytes", "cel_create", "cel_set_boundary", "cel_set_state",
           "cel_add_solitary", "cel_set_bathymetry", "cel_step", "cel_get_state", "cel_get_field",
           "cel_gauge_bytes", "cel_set_gauges", "cel_read_gauges", "cel_read_gauges_async", "cel_get_time",
           "cel_check_finite", "cel_checkpoint_bytes", "cel_save_checkpoint",
           "cel_load_checkpoint", "cel_runup_enable", "cel_render", "cel_adjoint_bytes",
           "cel_adjoint_gauge_misfit", "cel_adjoint_face_selfcheck", "cel_adjoint_input_gradient",
           "cel_get_stats", "cel_last_launch_count", "cel_profile_enable",
           "cel_profile_read", "cel_profile_disable", "cel_ensemble_table_bytes",
           "cel_ensemble_create", "cel_ensemble_step", "cel_ensemble_use_graphs", "cel_ensemble_graph_steps",
           "cel_ensemble_use_persistent", "cel_ensemble_persistent_steps", "cel_ensemble_check",
           "cel_ensemble_barrier_check", "cel_ensemble_last_launch_count",
           "cel_ensemble_profile_enable", "cel_ensemble_profile_read", "cel_ensemble_profile_disable",
           "cel_ensemble_last_error", "cel_ensemble_destroy", "cel_advance_noalloc", "cel_set_line_split",
           "cel_reset_line_splits", "cel_line_config", "cel_set_dependent_launch", "cel_get_dependent_launch",
           "cel_status_string",
           "cel_last_error", "cel_destroy"]


class CelGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("real_bytes", ctypes.c_int32)]


class CelParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("g", ctypes.c_double), ("Bdisp", ctypes.c_double),
                ("theta", ctypes.c_double), ("eps", ctypes.c_double), ("dt", ctypes.c_double),
                ("corrector_iters", ctypes.c_int32), ("still_water", ctypes.c_double),
                ("friction", ctypes.c_int32), ("fric_coef", ctypes.c_double)]


class CelBC(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("width_cells", ctypes.c_int32),
                ("ncomp", ctypes.c_int32), ("amp", ctypes.c_double * 8),
                ("period", ctypes.c_double * 8), ("theta", ctypes.c_double * 8),
                ("phase", ctypes.c_double * 8)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libceleris_gb.so (building it with nvcc when absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        d = ctypes.c_double
        L.cel_workspace_bytes.argtypes = [ctypes.POINTER(CelGrid), ctypes.POINTER(CelParams), ctypes.POINTER(sz)]
        L.cel_create.argtypes = [ctypes.POINTER(CelGrid), ctypes.POINTER(CelParams), vp, vp, sz, vp,
                                 ctypes.POINTER(vp)]
        L.cel_set_boundary.argtypes = [vp, i32, ctypes.POINTER(CelBC)]
        L.cel_set_state.argtypes = [vp, vp, vp, vp]
        L.cel_add_solitary.argtypes = [vp, d, d, d, d]
        L.cel_set_bathymetry.argtypes = [vp, vp]
        L.cel_step.argtypes = [vp, i32]
        L.cel_get_state.argtypes = [vp, vp, vp, vp]
        L.cel_get_field.argtypes = [vp, i32, vp]
        L.cel_gauge_bytes.argtypes = [i32, i32, i32, ctypes.POINTER(sz)]
        L.cel_set_gauges.argtypes = [vp, ctypes.POINTER(i32), i32, i32, i32, vp, sz]
        L.cel_read_gauges.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        L.cel_read_gauges_async.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        L.cel_get_time.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64)]
        L.cel_check_finite.argtypes = [vp]
        L.cel_checkpoint_bytes.argtypes = [vp, ctypes.POINTER(sz)]
        L.cel_save_checkpoint.argtypes = [vp, vp, sz]
        L.cel_load_checkpoint.argtypes = [vp, vp, sz]
        L.cel_runup_enable.argtypes = [vp, vp, d]
        L.cel_render.argtypes = [vp, ctypes.POINTER(CelRenderParams), vp]
        L.cel_adjoint_bytes.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(sz)]
        L.cel_adjoint_gauge_misfit.argtypes = [vp, i32, i32, ctypes.POINTER(i32), i32, vp, vp, sz, vp, vp, vp,
                                               ctypes.POINTER(d)]
        L.cel_adjoint_face_selfcheck.argtypes = [i32, vp, i32, vp, vp]
        L.cel_adjoint_input_gradient.argtypes = [vp, vp, vp]
        L.cel_get_stats.argtypes = [vp, ctypes.POINTER(CelStats)]
        L.cel_last_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
        L.cel_profile_enable.argtypes = [vp, i32]
        L.cel_profile_read.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64)]
        L.cel_profile_disable.argtypes = [vp]
        L.cel_advance_noalloc.argtypes = [ctypes.POINTER(CelGrid), ctypes.POINTER(CelParams),
                                          ctypes.POINTER(CelBC), vp, vp, vp, vp, vp, vp, vp, i32,
                                          i64, vp, ctypes.c_char_p, sz]
        L.cel_ensemble_table_bytes.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(sz)]
        L.cel_ensemble_create.argtypes = [ctypes.POINTER(vp), i32, vp, sz, vp, ctypes.POINTER(vp),
                                          ctypes.c_char_p, sz]
        L.cel_ensemble_step.argtypes = [vp, i32]
        L.cel_ensemble_use_graphs.argtypes = [vp, i32]
        L.cel_ensemble_graph_steps.argtypes = [vp, ctypes.POINTER(i64)]
        L.cel_ensemble_use_persistent.argtypes = [vp, i32, ctypes.c_double]
        L.cel_ensemble_persistent_steps.argtypes = [vp, ctypes.POINTER(i64)]
        L.cel_ensemble_check.argtypes = [vp]
        L.cel_ensemble_barrier_check.argtypes = [vp, i32, ctypes.c_double, ctypes.POINTER(i32)]
        L.cel_ensemble_last_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
        L.cel_ensemble_profile_enable.argtypes = [vp, i32]
        L.cel_ensemble_profile_read.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64)]
        L.cel_ensemble_profile_disable.argtypes = [vp]
        L.cel_set_line_split.argtypes = [i32, i32, i32]
        L.cel_reset_line_splits.argtypes = []
        L.cel_line_config.argtypes = [i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.cel_set_dependent_launch.argtypes = [i32]
        L.cel_get_dependent_launch.argtypes = [ctypes.POINTER(i32)]
        L.cel_ensemble_last_error.restype = ctypes.c_char_p
        L.cel_ensemble_last_error.argtypes = [vp]
        L.cel_ensemble_destroy.argtypes = [vp]
        L.cel_ensemble_destroy.restype = None
        L.cel_status_string.restype = ctypes.c_char_p
        L.cel_status_string.argtypes = [ctypes.c_int]
        L.cel_last_error.restype = ctypes.c_char_p
        L.cel_last_error.argtypes = [vp]
        L.cel_destroy.argtypes = [vp]
        L.cel_destroy.restype = None
        for name in EXPORTS:
            if name not in ("cel_status_string", "cel_last_error", "cel_destroy", "cel_ensemble_last_error",
                            "cel_ensemble_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


RENDER_MODES = {"eta": 0, "u": 1, "v": 2, "speed": 3, "fresnel": 4}


class CelStats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("max_speed", ctypes.c_double), ("wet_cells", ctypes.c_int64)]


class CelRenderParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("vmin", ctypes.c_float), ("vmax", ctypes.c_float),
                ("dry_h", ctypes.c_float), ("h_min", ctypes.c_float), ("zmin", ctypes.c_float),
                ("zmax", ctypes.c_float), ("grid", ctypes.c_float), ("exaggeration", ctypes.c_float),
                ("view", ctypes.c_float * 3), ("sun", ctypes.c_float * 3), ("absorb", ctypes.c_float)]


def render_params(mode="eta", vmin=-1.0, vmax=1.0, dry_h=1e-3, h_min=1e-2, zmin=-1.0, zmax=1.0, grid=0.0,
                  exaggeration=1.0, view=(0.0, 0.0, -1.0), sun=(0.3, 0.4, 1.0), absorb=0.5) -> CelRenderParams:
    return CelRenderParams(RENDER_MODES[mode] if isinstance(mode, str) else int(mode), vmin, vmax, dry_h, h_min,
                           zmin, zmax, grid, exaggeration, (ctypes.c_float * 3)(*view),
                           (ctypes.c_float * 3)(*sun), absorb)


class CelerisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def make_bc(type: int = SOLID, width: int = 0, comps: Sequence = ()) -> CelBC:
    """comps: (amp [m], period [s], direction [rad], phase [rad]) per component."""
    bc = CelBC()
    bc.type, bc.width_cells, bc.ncomp = int(type), int(width), len(comps)
    for m, (a, T, th, ph) in enumerate(comps):
        bc.amp[m], bc.period[m], bc.theta[m], bc.phase[m] = a, T, th, ph
    return bc


class Solver:
    """One simulation on one GPU.  Arrays in and out are torch tensors (ny, nx)."""

    def __init__(self, z, dx: float, dy: float, dt: float, *, dtype=None, model: int = BSNQ,
                 g: float = 9.81, Bd: float = 1.0 / 15.0, theta: float = 1.3, eps: float = 5e-12,
                 K: int = 0, ws: float = 0.0, friction: int = FRIC_NONE, fcoef: float = 0.0,
                 device=None, stream=None, poison: bool = False):
        """poison: fill the workspace with 0xFF bytes (NaN in every real
        field) before cel_create, so that a read of memory the library never
        wrote shows up as a non-finite state (a test aid)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the Celeris GB300 solver needs a CUDA device")
        self.torch = torch
        self.dtype = dtype or torch.float32
        if self.dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be float32 or float64")
        self.device = torch.device(device or "cuda")
        self.L = load()
        zt = torch.as_tensor(z).to(device=self.device, dtype=self.dtype).contiguous()
        self.ny, self.nx = zt.shape
        self.es = 4 if self.dtype == torch.float32 else 8
        self.grid = CelGrid(self.nx, self.ny, dx, dy, self.es)
        self.params = CelParams(model, g, Bd, theta, eps, dt, K, ws, friction, fcoef)
        nb = ctypes.c_size_t()
        self._check(self.L.cel_workspace_bytes(ctypes.byref(self.grid), ctypes.byref(self.params),
                                               ctypes.byref(nb)), "workspace_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
            if poison:
                self.workspace.fill_(255)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        h = ctypes.c_void_p()
        self._h = None
        st = self.L.cel_create(ctypes.byref(self.grid), ctypes.byref(self.params), zt.data_ptr(),
                               self._ws_ptr, nb.value, self.stream.cuda_stream, ctypes.byref(h))
        if st != CEL_OK:
            raise CelerisError(st, "cel_create failed")
        self._h = h
        self._z = zt
        self._gauge_buf = None
        self.ng = 0

    # ------------------------------------------------------------ plumbing
    def _check(self, st: int, what: str):
        if st != CEL_OK:
            msg = ""
            if getattr(self, "_h", None):
                msg = self.L.cel_last_error(self._h).decode()
            raise CelerisError(st, f"{what}: {msg}")

    def _arr(self, a):
        t = self.torch.as_tensor(a).to(device=self.device, dtype=self.dtype).contiguous()
        if t.shape != (self.ny, self.nx):
            raise ValueError(f"expected shape {(self.ny, self.nx)}, got {tuple(t.shape)}")
        return t

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self.L.cel_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- calls
    def set_boundary(self, side: int, type: int = SOLID, width: int = 0, comps: Sequence = ()):
        bc = make_bc(type, width, comps)
        self._check(self.L.cel_set_boundary(self._h, side, ctypes.byref(bc)), "set_boundary")

    def set_state(self, w, P, Q):
        w, P, Q = self._arr(w), self._arr(P), self._arr(Q)
        self._check(self.L.cel_set_state(self._h, w.data_ptr(), P.data_ptr(), Q.data_ptr()), "set_state")
        self.stream.synchronize()

    def add_solitary(self, H: float, theta: float, x0: float, y0: float):
        self._check(self.L.cel_add_solitary(self._h, H, theta, x0, y0), "add_solitary")

    def set_bathymetry(self, z):
        zt = self._arr(z)
        self._check(self.L.cel_set_bathymetry(self._h, zt.data_ptr()), "set_bathymetry")
        self.stream.synchronize()

    def step(self, n: int = 1):
        self._check(self.L.cel_step(self._h, int(n)), "step")

    def state(self) -> Tuple:
        t = self.torch
        w = t.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        P, Q = t.empty_like(w), t.empty_like(w)
        self._check(self.L.cel_get_state(self._h, w.data_ptr(), P.data_ptr(), Q.data_ptr()), "get_state")
        self.stream.synchronize()
        return w, P, Q

    def stats(self) -> dict:
        """Mass [m^3], largest speed [m/s] and wet-cell count of the present
        state (cel_get_stats)."""
        st = CelStats()
        self._check(self.L.cel_get_stats(self._h, ctypes.byref(st)), "get_stats")
        return {"mass": st.mass, "max_speed": st.max_speed, "wet_cells": st.wet_cells}

    def field(self, name: str):
        out = self.torch.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        self._check(self.L.cel_get_field(self._h, FIELDS[name], out.data_ptr()), "get_field")
        self.stream.synchronize()
        return out

    def set_gauges(self, ij, log_every: int, capacity: int):
        ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
        nb = ctypes.c_size_t()
        self._check(self.L.cel_gauge_bytes(len(ij), capacity, self.es, ctypes.byref(nb)), "gauge_bytes")
        buf = self.torch.empty(nb.value + 256, dtype=self.torch.uint8, device=self.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        self._check(self.L.cel_set_gauges(self._h, ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          len(ij), log_every, capacity, ptr, nb.value), "set_gauges")
        self.stream.synchronize()
        self._gauge_buf = buf
        self.ng = len(ij)

    def read_gauges(self, max_rec: int) -> np.ndarray:
        out = np.zeros((max_rec, self.ng), dtype=np.float32 if self.es == 4 else np.float64)
        n = ctypes.c_int32()
        self._check(self.L.cel_read_gauges(self._h, out.ctypes.data, max_rec, ctypes.byref(n)), "read_gauges")
        return out[: n.value]

    def read_gauges_async(self, out) -> int:
        """Queue the copy of up to len(out) oldest gauge records into `out`
        (a pinned host tensor [records, gauges] of the solver's dtype) on the
        solver's stream without synchronising (cel_read_gauges_async);
        returns the records queued.  The values are there once the stream has
        passed this point."""
        if out.device.type != "cpu" or out.dim() != 2 or out.shape[1] != self.ng or not out.is_contiguous():
            raise ValueError("out must be a contiguous host tensor [records, gauges]")
        if out.element_size() != self.es:
            raise ValueError("out must have the solver's precision")
        n = ctypes.c_int32()
        self._check(self.L.cel_read_gauges_async(self._h, out.data_ptr(), out.shape[0], ctypes.byref(n)),
                    "read_gauges_async")
        return n.value

    def time(self):
        t, s = ctypes.c_double(), ctypes.c_int64()
        self._check(self.L.cel_get_time(self._h, ctypes.byref(t), ctypes.byref(s)), "get_time")
        return t.value, s.value

    def check_finite(self) -> bool:
        st = self.L.cel_check_finite(self._h)
        if st == 4:
            return False
        self._check(st, "check_finite")
        return True

    def checkpoint(self):
        nb = ctypes.c_size_t()
        self._check(self.L.cel_checkpoint_bytes(self._h, ctypes.byref(nb)), "checkpoint_bytes")
        buf = self.torch.empty(nb.value, dtype=self.torch.uint8, device=self.device)
        self._check(self.L.cel_save_checkpoint(self._h, buf.data_ptr(), nb.value), "save_checkpoint")
        self.stream.synchronize()
        return buf

    def restore(self, buf):
        self._check(self.L.cel_load_checkpoint(self._h, buf.data_ptr(), buf.numel()), "load_checkpoint")
        self.stream.synchronize()

    def profile_enable(self, capacity: int):
        self._check(self.L.cel_profile_enable(self._h, int(capacity)), "profile_enable")

    def profile_read(self):
        """{kernel: (total ms, launches)} since enable or the last read."""
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        self._check(self.L.cel_profile_read(self._h, ms, cnt), "profile_read")
        return {name: (ms[k], cnt[k]) for k, name in enumerate(("stencil", "lines", "ghosts"))}

    def profile_disable(self):
        self._check(self.L.cel_profile_disable(self._h), "profile_disable")

    def last_launch_count(self) -> int:
        n = ctypes.c_int64()
        self._check(self.L.cel_last_launch_count(self._h, ctypes.byref(n)), "last_launch_count")
        return n.value

    def render(self, params: Optional[CelRenderParams] = None, out=None, **kw):
        """RGBA image (ny, nx, 4) uint8 on the device of the present state
        (row j = grid row j); params from render_params(...) or keywords."""
        p = params if params is not None else render_params(**kw)
        if out is None:
            with self.torch.cuda.device(self.device):
                out = self.torch.empty((self.ny, self.nx, 4), dtype=self.torch.uint8, device=self.device)
        self._check(self.L.cel_render(self._h, ctypes.byref(p), out.data_ptr()), "render")
        return out

    def runup_enable(self, delta: float):
        """Track the highest w seen where the depth exceeds delta (Sec. 4.1,
        4.3), from the present state on; the field lives in a tensor this
        object keeps."""
        with self.torch.cuda.device(self.device):
            self._runup = self.torch.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        self._check(self.L.cel_runup_enable(self._h, self._runup.data_ptr(), float(delta)), "runup_enable")

    def runup_disable(self):
        self._check(self.L.cel_runup_enable(self._h, None, 0.0), "runup_disable")
        self._runup = None

    def runup(self):
        """(ny, nx) highest w seen while wetter than the threshold, -inf where
        never (a copy, after the stream's work so far)."""
        if getattr(self, "_runup", None) is None:
            raise CelerisError(1, "run-up tracking is not enabled")
        self.stream.synchronize()
        return self._runup.clone()


class Ensemble:
    """Many Solvers of one precision and one K, stepped in lockstep with one
    launch per kernel kind and stage (cel_ensemble_*).  The members stay
    usable alone (state, fields, gauges, checkpoints) between ensemble steps;
    the ensemble keeps them alive.  Its launches go to ``stream`` (the current
    stream by default).  poison: fill the argument tables with 0xFF bytes
    before cel_ensemble_create (a test aid, as for Solver)."""

    def __init__(self, members: Sequence[Solver], stream=None, poison: bool = False):
        torch = members[0].torch
        self.torch = torch
        self.members = list(members)
        self.L = load()
        n = len(self.members)
        hs = (ctypes.c_void_p * n)(*[m._h.value for m in self.members])
        nb = ctypes.c_size_t()
        st = self.L.cel_ensemble_table_bytes(hs, n, ctypes.byref(nb))
        if st != CEL_OK:
            raise CelerisError(st, "cel_ensemble_table_bytes failed (mixed precision or K, shared workspace)")
        dev = self.members[0].device
        with torch.cuda.device(dev):
            self.stream = stream or torch.cuda.current_stream(dev)
            self.table = torch.empty(nb.value + 256, dtype=torch.uint8, device=dev)
            if poison:
                self.table.fill_(255)
        ptr = (self.table.data_ptr() + 255) // 256 * 256
        msg = ctypes.create_string_buffer(256)
        h = ctypes.c_void_p()
        self._h = None
        st = self.L.cel_ensemble_create(hs, n, ptr, nb.value, self.stream.cuda_stream, ctypes.byref(h), msg,
                                        len(msg))
        if st != CEL_OK:
            raise CelerisError(st, msg.value.decode())
        self._h = h

    def step(self, n: int = 1):
        st = self.L.cel_ensemble_step(self._h, int(n))
        if st != CEL_OK:
            raise CelerisError(st, self.L.cel_ensemble_last_error(self._h).decode())

    def use_graphs(self, enable: bool = True):
        """Replay captured 6-step cycles (the default) or launch every step
        kernel by kernel (cel_ensemble_use_graphs)."""
        st = self.L.cel_ensemble_use_graphs(self._h, int(bool(enable)))
        if st != CEL_OK:
            raise CelerisError(st, "cel_ensemble_use_graphs failed")

    def use_persistent(self, enable: bool = True, timeout_ms: float = 1000.0):
        """Take each call's steps in one persistent cooperative launch where
        the captured cycle's conditions hold (cel_ensemble_use_persistent);
        every grid-wide wait is bounded by timeout_ms."""
        st = self.L.cel_ensemble_use_persistent(self._h, int(bool(enable)), float(timeout_ms))
        if st != CEL_OK:
            raise CelerisError(st, self.L.cel_ensemble_last_error(self._h).decode())

    def persistent_steps(self) -> int:
        """Steps taken by persistent launches since creation."""
        v = ctypes.c_int64()
        self.L.cel_ensemble_persistent_steps(self._h, ctypes.byref(v))
        return v.value

    def check(self):
        """Synchronise; raises CelerisError (CEL_ERR_TIMEOUT) if a wait of a
        persistent launch ran out."""
        st = self.L.cel_ensemble_check(self._h)
        if st != CEL_OK:
            raise CelerisError(st, self.L.cel_ensemble_last_error(self._h).decode())

    def barrier_check(self, missing: int, timeout_ms: float) -> bool:
        """One persistent launch of a single barrier that expects `missing`
        more blocks than run; True if its wait ran out."""
        v = ctypes.c_int32()
        st = self.L.cel_ensemble_barrier_check(self._h, int(missing), float(timeout_ms), ctypes.byref(v))
        if st != CEL_OK:
            raise CelerisError(st, self.L.cel_ensemble_last_error(self._h).decode())
        return bool(v.value)

    def last_launch_count(self) -> int:
        v = ctypes.c_int64()
        self.L.cel_ensemble_last_launch_count(self._h, ctypes.byref(v))
        return v.value

    def graph_steps(self) -> int:
        """Steps taken by replaying a captured 6-step cycle since creation."""
        v = ctypes.c_int64()
        self.L.cel_ensemble_graph_steps(self._h, ctypes.byref(v))
        return v.value

    def profile_enable(self, capacity: int):
        st = self.L.cel_ensemble_profile_enable(self._h, int(capacity))
        if st != CEL_OK:
            raise CelerisError(st, self.L.cel_ensemble_last_error(self._h).decode())

    def profile_read(self):
        """{kernel: (ms summed, launches)} for 'stencil', 'lines', 'ghosts'."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        st = self.L.cel_ensemble_profile_read(self._h, ms, n)
        if st != CEL_OK:
            raise CelerisError(st, self.L.cel_ensemble_last_error(self._h).decode())
        return {k: (ms[i], n[i]) for i, k in enumerate(("stencil", "lines", "ghosts"))}

    def profile_disable(self):
        self.L.cel_ensemble_profile_disable(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.stream.synchronize()   # its launches read the argument tables this object owns
            self.L.cel_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_line_split(real_bytes: int, max_rows: int, rows_per_thread: int):
    """The line solver's rows per thread for lines of up to max_rows rows
    (cel_set_line_split; 0 removes the class)."""
    st = load().cel_set_line_split(int(real_bytes), int(max_rows), int(rows_per_thread))
    if st != CEL_OK:
        raise CelerisError(st, "cel_set_line_split: bad size or rows per thread")


def reset_line_splits():
    """Back to the built-in rule (cel_reset_line_splits)."""
    load().cel_reset_line_splits()


def set_dependent_launch(enable: bool = True):
    """Programmatic dependent launch of the step's kernels (process-wide;
    cel_set_dependent_launch).  The results do not depend on it."""
    load().cel_set_dependent_launch(int(bool(enable)))


def dependent_launch() -> bool:
    v = ctypes.c_int32()
    load().cel_get_dependent_launch(ctypes.byref(v))
    return bool(v.value)


def line_config(real_bytes: int, rows: int):
    """(rows per thread, threads per block) of a line of `rows` rows."""
    m, t = ctypes.c_int32(), ctypes.c_int32()
    st = load().cel_line_config(int(real_bytes), int(rows), ctypes.byref(m), ctypes.byref(t))
    if st != CEL_OK:
        raise CelerisError(st, "cel_line_config: bad size")
    return m.value, t.value


def adjoint_scratch_bytes(solver: "Solver", nsteps: int, ngauges: int, ckpt_every: int = 100,
                          bed: bool = False) -> int:
    """Bytes of the scratch tensor gauge_misfit_gradient needs (the
    cel_adjoint_bytes figure plus 256 for alignment)."""
    nb = ctypes.c_size_t()
    solver._check(solver.L.cel_adjoint_bytes(solver._h, nsteps, ckpt_every, ngauges, int(bed), ctypes.byref(nb)),
                  "adjoint_bytes")
    return nb.value + 256


def gauge_misfit_gradient(solver: "Solver", nsteps: int, gauges, obs, ckpt_every: int = 100, bed: bool = False,
                          poison: bool = False, scratch=None):
    """Run nsteps from the solver's present (freshly set) state and return
    (L, eta, dL/dw0), plus dL/dz when bed is set: the gauge misfit
    L = 1/2 sum (eta - obs)^2 over steps 1..nsteps, the recorded eta
    ([nsteps, ngauges] tensor) and its gradients with respect to w at the
    start and to the cell-centre bed ([ny, nx] tensors), by the discrete
    adjoint (cel_adjoint_gauge_misfit).  obs: [nsteps, ngauges].
    ckpt_every: checkpoint spacing of the recomputation; 0 keeps every step
    of the forward run instead (no recomputation; the scratch grows with
    nsteps).  scratch: a uint8 CUDA tensor of at least
    adjoint_scratch_bytes(...) bytes to use (else one is allocated).
    poison: fill the scratch with 0xFF bytes first (a test aid, as for
    Solver)."""
    torch = solver.torch
    ij = np.ascontiguousarray(np.asarray(gauges, dtype=np.int32).reshape(-1, 2))
    ng = len(ij)
    obs_t = torch.as_tensor(obs).to(device=solver.device, dtype=solver.dtype).contiguous()
    if tuple(obs_t.shape) != (nsteps, ng):
        raise ValueError("obs must be [nsteps, ngauges]")
    need = adjoint_scratch_bytes(solver, nsteps, ng, ckpt_every, bed)
    nb = ctypes.c_size_t(need - 256)
    with torch.cuda.device(solver.device):
        if scratch is None:
            scratch = torch.empty(need, dtype=torch.uint8, device=solver.device)
        elif (scratch.dtype != torch.uint8 or not scratch.is_cuda or scratch.numel() < need
              or scratch.get_device() != torch.cuda.current_device()):
            raise ValueError(f"scratch must be a uint8 tensor of at least {need} bytes on the solver's device")
        if poison:
            scratch.fill_(255)
        eta = torch.empty((nsteps, ng), dtype=solver.dtype, device=solver.device)
        grad = torch.empty((solver.ny, solver.nx), dtype=solver.dtype, device=solver.device)
        grad_z = torch.empty((solver.ny, solver.nx), dtype=solver.dtype, device=solver.device) if bed else None
    ptr = (scratch.data_ptr() + 255) // 256 * 256
    loss = ctypes.c_double()
    st = solver.L.cel_adjoint_gauge_misfit(solver._h, nsteps, ckpt_every,
                                           ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ng,
                                           obs_t.data_ptr(), ptr, nb.value, eta.data_ptr(), grad.data_ptr(),
                                           grad_z.data_ptr() if bed else None, ctypes.byref(loss))
    solver._check(st, "adjoint_gauge_misfit")
    return (loss.value, eta, grad, grad_z) if bed else (loss.value, eta, grad)


def face_vjp_selfcheck(inputs):
    """The adjoint's face-flux VJP by dual numbers and by hand on the faces
    in `inputs` ([n, 22] device tensor, float32 or float64; the column order
    of cel_adjoint_face_selfcheck).  Returns ([n, 15], [n, 15])."""
    import torch
    x = inputs.contiguous()
    if x.dim() != 2 or x.shape[1] != 22 or x.dtype not in (torch.float32, torch.float64) or not x.is_cuda:
        raise ValueError("inputs must be an [n, 22] float32/float64 CUDA tensor")
    out = torch.empty((x.shape[0], 30), dtype=x.dtype, device=x.device)
    lib = load()
    st = lib.cel_adjoint_face_selfcheck(x.element_size(), x.data_ptr(), x.shape[0], out.data_ptr(),
                                        torch.cuda.current_stream(x.device).cuda_stream)
    if st != 0:
        raise CelerisError(f"face_vjp_selfcheck failed ({st})")
    return out[:, :15], out[:, 15:]


def _gauge_misfit_function():
    import torch

    class GaugeMisfit(torch.autograd.Function):
        """L(w0, z) = 1/2 sum (eta - obs)^2 over nsteps steps from w0 (with P0,
        Q0 fixed) over the bed z (None: the solver's bed, not differentiated);
        backward gives dL/dw0 and dL/dz from the discrete adjoint.  Where w0
        lies below the bed the state is clamped to it: the gradient in w0 is
        0 there, and w follows the bed."""

        @staticmethod
        def forward(ctx, w0, z, solver, P0, Q0, nsteps, gauges, obs, ckpt_every=100):
            if z is not None:
                solver.set_bathymetry(z)
            solver.set_state(w0, P0, Q0)
            out = gauge_misfit_gradient(solver, nsteps, gauges, obs, ckpt_every, bed=z is not None)
            loss, grad = out[0], out[2]
            w_in = w0.to(device=grad.device, dtype=grad.dtype).contiguous()
            solver._check(solver.L.cel_adjoint_input_gradient(solver._h, w_in.data_ptr(), grad.data_ptr()),
                          "adjoint_input_gradient")
            grad_z = out[3] if z is not None else torch.zeros_like(grad)
            ctx.has_z = z is not None
            ctx.save_for_backward(grad, grad_z)
            return torch.tensor(loss, dtype=w0.dtype, device=w0.device)

        @staticmethod
        def backward(ctx, gout):
            grad, grad_z = ctx.saved_tensors
            gz = (grad_z * gout).to(gout.dtype) if ctx.has_z else None
            return (grad * gout).to(gout.dtype), gz, None, None, None, None, None, None, None

    return GaugeMisfit


def gauge_misfit(w0, solver, P0, Q0, nsteps, gauges, obs, ckpt_every=100, z=None):
    """Differentiable gauge misfit (torch.autograd) of a run from w0, and
    over the bed z when one is given."""
    return _gauge_misfit_function().apply(w0, z, solver, P0, Q0, nsteps, gauges, obs, ckpt_every)


def ensemble_share(cells: Sequence[int], rank: Optional[int] = None, world: Optional[int] = None) -> list:
    """Indices of the scenarios one rank steps when an ensemble is sharded
    over ranks (one GPU each, no data exchanged between them): the split of
    scenarios.partition, largest first to the rank with the fewest cells.
    cells: the scenarios' cell counts.  rank and world default to those of
    torch.distributed when it is initialised, else 0 and 1."""
    from . import scenarios as _sc
    if rank is None or world is None:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            rank, world = dist.get_rank(), dist.get_world_size()
        else:
            rank, world = 0, 1
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return _sc.partition(list(cells), world)[rank]


def sharded_ensemble(scenarios, dtype=None, rank: Optional[int] = None, world: Optional[int] = None,
                     stream=None, **kw):
    """This rank's share of an ensemble sharded over ranks: (Ensemble of its
    members, the scenarios' indices).  Each rank steps its share alone; the
    members' results do not depend on the sharding."""
    share = ensemble_share([s.cells for s in scenarios], rank, world)
    members = [from_scenario(scenarios[k], dtype=dtype, **kw) for k in share]
    return Ensemble(members, stream=stream), share


def from_scenario(s, dtype=None, K: Optional[int] = None, **kw) -> Solver:
    """A Solver set up with a scenario's bed, boundaries, state and solitons."""
    sol = Solver(s.z, s.dx, s.dy, s.dt, dtype=dtype, model=s.model, g=s.g, Bd=s.Bd, theta=s.theta,
                 eps=s.eps, K=s.K if K is None else K, ws=s.ws, friction=s.friction, fcoef=s.fcoef, **kw)
    for side, sd in s.sides.items():
        sol.set_boundary(side, sd.type, sd.width, sd.comps)
    sol.set_state(*s.initial_state())
    for (H, th, x0, y0) in s.solitons:
        sol.add_solitary(H, th, x0, y0)
    return sol
