"""The C-ABI library builds, loads and exports every entry point the header
declares (no compute calls: no GPU here).  Host-only calls are exercised."""
import ctypes
import os
import re

import pytest

from paper_1611_05984_gb300 import build as cbuild
from paper_1611_05984_gb300 import celeris

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "celeris_gb.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cel_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    try:
        path = cbuild.build()
    except (RuntimeError, FileNotFoundError) as e:   # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"missing export {n}"
    assert sorted(celeris.EXPORTS) == names


def test_workspace_bytes_and_validation():
    L = celeris.load()
    g = celeris.CelGrid(2048, 2048, 1.0, 1.0, 4)
    p = celeris.CelParams(0, 9.81, 1 / 15, 1.3, 5e-12, 0.01, 1, 0.0, 2, 0.015)
    nb = ctypes.c_size_t()
    assert L.cel_workspace_bytes(ctypes.byref(g), ctypes.byref(p), ctypes.byref(nb)) == 0
    # 24 row-major fields (w and P twice, dU*, d, AB3 and AM4 carries), 4
    # column-major fields (Q twice, dV*, d) and the bed corners, each 2048^2
    # floats, plus the dry-cell masks
    assert 29 * 2048 * 2048 * 4 <= nb.value < 30 * 2048 * 2048 * 4
    p0 = celeris.CelParams(0, 9.81, 1 / 15, 1.3, 5e-12, 0.01, 0, 0.0, 2, 0.015)
    nb0 = ctypes.c_size_t()
    assert L.cel_workspace_bytes(ctypes.byref(g), ctypes.byref(p0), ctypes.byref(nb0)) == 0
    assert nb0.value < nb.value
    for bad in (celeris.CelGrid(1, 8, 1.0, 1.0, 4), celeris.CelGrid(8, 8, 0.0, 1.0, 4),
                celeris.CelGrid(8, 8, 1.0, 1.0, 2), celeris.CelGrid(20000, 8, 1.0, 1.0, 4),
                celeris.CelGrid(9000, 8, 1.0, 1.0, 8)):
        assert L.cel_workspace_bytes(ctypes.byref(bad), ctypes.byref(p), ctypes.byref(nb)) == 1
    for badp in (celeris.CelParams(2, 9.81, 1 / 15, 1.3, 5e-12, 0.01, 0, 0.0, 0, 0.0),
                 celeris.CelParams(0, 9.81, 1 / 15, 1.3, 5e-12, -1.0, 0, 0.0, 0, 0.0),
                 celeris.CelParams(0, 9.81, 1 / 15, 3.0, 5e-12, 0.01, 0, 0.0, 0, 0.0),
                 celeris.CelParams(0, 9.81, 1 / 15, 1.3, 5e-12, 0.01, -1, 0.0, 0, 0.0)):
        assert L.cel_workspace_bytes(ctypes.byref(g), ctypes.byref(badp), ctypes.byref(nb)) == 1
    assert L.cel_gauge_bytes(4, 10, 4, ctypes.byref(nb)) == 0 and nb.value >= 4 * 10 * 4
    assert L.cel_status_string(4) == b"non-finite value in the state"
    assert L.cel_last_error(None) == b""


def test_create_rejects_bad_arguments_without_gpu_work():
    L = celeris.load()
    g = celeris.CelGrid(64, 64, 1.0, 1.0, 4)
    p = celeris.CelParams(0, 9.81, 1 / 15, 1.3, 5e-12, 0.01, 0, 0.0, 0, 0.0)
    h = ctypes.c_void_p()
    # NULL bed / workspace, misaligned workspace, too-small workspace: all
    # rejected before any CUDA call is made
    assert L.cel_create(ctypes.byref(g), ctypes.byref(p), None, 256, 1 << 30, None, ctypes.byref(h)) == 1
    assert L.cel_create(ctypes.byref(g), ctypes.byref(p), 256, None, 1 << 30, None, ctypes.byref(h)) == 1
    assert L.cel_create(ctypes.byref(g), ctypes.byref(p), 256, 257, 1 << 30, None, ctypes.byref(h)) == 1
    assert L.cel_create(ctypes.byref(g), ctypes.byref(p), 256, 512, 16, None, ctypes.byref(h)) == 2
    assert not h.value


def test_ensemble_rejects_empty_member_lists_without_gpu_work():
    lib = celeris.load()
    nb = ctypes.c_size_t(123)
    assert lib.cel_ensemble_table_bytes(None, 0, ctypes.byref(nb)) == 1
    assert nb.value == 123
    out = ctypes.c_void_p()
    msg = ctypes.create_string_buffer(128)
    assert lib.cel_ensemble_create(None, 0, None, 0, None, ctypes.byref(out), msg, len(msg)) == 1
    assert out.value is None
    assert b"at least one member" in msg.value
    arr = (ctypes.c_void_p * 2)(None, None)
    assert lib.cel_ensemble_table_bytes(arr, 2, ctypes.byref(nb)) == 1
    assert lib.cel_ensemble_step(None, 1) == 1
    assert lib.cel_ensemble_last_error(None) == b""
    lib.cel_ensemble_destroy(None)


def test_adjoint_entry_points_reject_bad_arguments_without_gpu_work():
    """The adjoint's calls validate on the host before any device work: a
    NULL solver, non-positive step or gauge counts, a negative checkpoint
    spacing, and the
    face self-check's element size and counts."""
    L = celeris.load()
    nb = ctypes.c_size_t()
    assert L.cel_adjoint_bytes(None, 10, 5, 4, 1, ctypes.byref(nb)) == 1
    loss = ctypes.c_double()
    assert L.cel_adjoint_gauge_misfit(None, 10, 5, None, 4, None, None, 0, None, None, None,
                                      ctypes.byref(loss)) == 1
    assert L.cel_adjoint_face_selfcheck(3, None, 4, None, None) == 1     # element size 4 or 8
    assert L.cel_adjoint_face_selfcheck(4, None, -1, None, None) == 1    # a negative count
    assert L.cel_adjoint_face_selfcheck(8, None, 5, None, None) == 1     # NULL buffers
    assert L.cel_adjoint_face_selfcheck(4, None, 0, None, None) == 0     # nothing to do


def test_line_split_table():
    """The line solver's split per class of line lengths (cel_set_line_split,
    the autotuner's setting): the built-in rule, a class overriding it where
    the block fits, removal, reset, and the argument checks.  Host logic."""
    L = celeris.load()
    celeris.reset_line_splits()
    try:
        assert celeris.line_config(4, 50) == (2, 32)
        assert celeris.line_config(4, 100) == (4, 32)
        assert celeris.line_config(4, 2048) == (8, 256)
        assert celeris.line_config(4, 8192) == (8, 1024)
        assert celeris.line_config(8, 4096) == (8, 512)
        celeris.set_line_split(4, 256, 4)          # lines of 129..256 rows: 4 rows per thread
        assert celeris.line_config(4, 200) == (4, 64)
        assert celeris.line_config(4, 100) == (4, 32)   # below the class: the same class (the first that fits)
        assert celeris.line_config(4, 300) == (8, 64)   # above it: the built-in rule
        assert celeris.line_config(8, 200) == (8, 32)   # the other precision is untouched
        celeris.set_line_split(4, 8192, 2)         # 4096 threads would not fit: the built-in rule
        assert celeris.line_config(4, 8192) == (8, 1024)
        assert celeris.line_config(4, 300) == (2, 160)  # where it fits, the class 257..8192 applies
        celeris.set_line_split(4, 256, 0)          # removed: lines of 200 rows fall in the 8192 class
        assert celeris.line_config(4, 200) == (2, 128)
        celeris.set_line_split(4, 8192, 0)
        assert celeris.line_config(4, 200) == (8, 32)
        with pytest.raises(celeris.CelerisError):
            celeris.set_line_split(4, 256, 3)
        with pytest.raises(celeris.CelerisError):
            celeris.set_line_split(2, 256, 4)
        with pytest.raises(celeris.CelerisError):
            celeris.line_config(4, 20000)
    finally:
        celeris.reset_line_splits()
    assert celeris.line_config(4, 200) == (8, 32)


def test_launch_switch_and_queued_reads_without_gpu_work():
    """The dependent-launch switch (on by default) reads back what was set;
    the queued gauge read and the persistent ensemble's calls refuse NULL
    handles and out-pointers before any CUDA call, leaving the outputs
    untouched."""
    L = celeris.load()
    v = ctypes.c_int32(-1)
    assert L.cel_get_dependent_launch(ctypes.byref(v)) == 0
    old = v.value
    assert old in (0, 1)
    try:
        for want in (0, 1, 0):
            assert L.cel_set_dependent_launch(want) == 0
            assert L.cel_get_dependent_launch(ctypes.byref(v)) == 0 and v.value == want
        assert L.cel_set_dependent_launch(5) == 0                   # any non-zero value turns it on
        assert L.cel_get_dependent_launch(ctypes.byref(v)) == 0 and v.value == 1
    finally:
        L.cel_set_dependent_launch(old)
    assert L.cel_get_dependent_launch(None) == 1
    n = ctypes.c_int32(7)
    assert L.cel_read_gauges_async(None, None, 0, ctypes.byref(n)) == 1 and n.value == 7
    assert L.cel_ensemble_use_persistent(None, 1, 100.0) == 1
    steps = ctypes.c_int64(5)
    assert L.cel_ensemble_persistent_steps(None, ctypes.byref(steps)) == 1 and steps.value == 5
    assert L.cel_ensemble_check(None) == 1
    t = ctypes.c_int32(3)
    assert L.cel_ensemble_barrier_check(None, 0, 10.0, ctypes.byref(t)) == 1 and t.value == 3
