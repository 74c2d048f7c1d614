"""CPU-only checks of the C ABI: the library loads, exports every function
include/xs_api.h declares, rejects bad arguments before touching a GPU, and
its host-side ring layout (used by the XSVS contrast) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2204_13241_gb300 import _native as nat
from paper_2204_13241_gb300 import build as xbuild
from paper_2204_13241_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    xbuild.build()
    return nat.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "xs_api.h")).read()
    return sorted(set(re.findall(r"^XS_API\s+[\w\s\*]+?\b(xs_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("xs_intensity", "xs_g2", "xs_xsvs_contrast", "xs_intensity_backward"):
        assert must in names
    assert sorted(nat.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", nat.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(xs_\w+)", out))
    assert set(_declared()) <= exported
    for name in _declared():
        assert hasattr(lib, name)


def test_null_arguments_are_rejected_without_a_gpu(lib):
    assert lib.xs_intensity(None, None, None, 0, None, None, None) == 1
    assert "required" in lib.xs_last_error().decode()
    assert lib.xs_g2(None, None, 1, 1, None, 0, None, None, None) == 1
    assert lib.xs_intensity_backward(None, None, None, None, None, None, None) == 1
    assert lib.xs_context_destroy(None) == 0
    assert lib.xs_version().decode().startswith("xs")


def test_context_creation_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.xs_context_create(None, ctypes.byref(h))
    assert st == 4 and not h.value
    assert "device" in lib.xs_last_error().decode().lower()


@pytest.mark.parametrize("side,width", [(64, 1.0), (33, 1.0), (40, 0.55)])
def test_ring_layout_matches_oracle(lib, side, width):
    grid = wl.QGrid(-(side // 2), side, -(side // 3), side, 0, 1)
    L = 37.0
    box = np.eye(3) * L
    n_rings = wl.rings_for_plane(grid)
    g = nat.QGrid(*grid.as_tuple())
    b = nat.Box()
    for i, v in enumerate(box.reshape(-1)):
        b.h[i] = v
    out = np.zeros(grid.n_pixels, dtype=np.int32)
    assert lib.xs_ring_index(ctypes.byref(g), ctypes.byref(b), width, n_rings,
                             out.ctypes.data_as(ctypes.c_void_p)) == 0
    ref = oracle.ring_index(box, grid.miller(), width, n_rings)
    assert np.array_equal(out, ref)


def test_ring_layout_rejects_bad_width(lib):
    g = nat.QGrid(-4, 8, -4, 8, 0, 1)
    b = nat.Box()
    for i, v in enumerate(np.eye(3).reshape(-1) * 10):
        b.h[i] = v
    out = np.zeros(64, dtype=np.int32)
    assert lib.xs_ring_index(ctypes.byref(g), ctypes.byref(b), 1.5, 5, out.ctypes.data_as(ctypes.c_void_p)) == 1
    sing = nat.Box()
    assert lib.xs_ring_index(ctypes.byref(g), ctypes.byref(sing), 1.0, 5, out.ctypes.data_as(ctypes.c_void_p)) == 1


def test_triclinic_ring_layout_matches_oracle(lib):
    grid = wl.QGrid(-6, 13, -5, 11, -2, 5)
    box = np.array([[12.0, 3.0, -1.5], [0.0, 10.0, 2.5], [1.0, 0.0, 9.0]])
    g = nat.QGrid(*grid.as_tuple())
    b = nat.Box()
    for i, v in enumerate(box.reshape(-1)):
        b.h[i] = v
    out = np.zeros(grid.n_pixels, dtype=np.int32)
    assert lib.xs_ring_index(ctypes.byref(g), ctypes.byref(b), 1.0, 9, out.ctypes.data_as(ctypes.c_void_p)) == 0
    ref = oracle.ring_index(box, grid.miller(), 1.0, 9)
    assert np.array_equal(out, ref)


def test_ewald_points_host_helper_matches_oracle():
    # host-side library helper (no GPU work) against the oracle's selection
    import math
    from paper_2204_13241_gb300 import api as xs
    cases = [(np.eye(3) * 40.0, [0.0, 0.0, 2 * math.pi / 1.3], (-40, 80, -36, 72)),
             (np.array([[30.0, 4.0, -2.0], [0.0, 27.0, 3.0], [0.0, 0.0, 33.0]]), [0.3, -0.2, 8.0], (-20, 40, -24, 48)),
             (np.eye(3) * 25.0, [1.0, 0.0, 0.0], (-8, 16, -8, 16))]
    for box, k, win in cases:
        m1, v1 = xs.ewald_points(box, k, *win)
        m2, v2 = oracle.ewald_points(box, k, *win)
        assert np.array_equal(v1, v2)
        assert np.array_equal(m1[v1], m2[v2])


def test_static_entry_rejects_bad_arguments_before_any_launch(lib):
    # the allocation-free entry applies xs_intensity's checks: grid extents,
    # atom count and memory kind of every pointer a kernel would dereference;
    # host buffers are refused with XS_ERR_INVALID_ARG instead of reaching a
    # kernel (on a machine without a GPU every buffer counts as host memory)
    from paper_2204_13241_gb300 import api
    pos = np.zeros((2, 10, 3), np.float32)
    f = np.ones(10, np.float32)
    I = np.zeros((2, 1, 8, 8), np.float32)
    tr = nat.Traj(pos.ctypes.data, 0, f.ctypes.data, 10, 2, api._box(np.eye(3) * 10.0))
    g = nat.QGrid(-4, 8, -4, 8, 0, 1)
    st = lib.xs_intensity_fp32_static(ctypes.byref(tr), ctypes.byref(g), I.ctypes.data, None, None, None)
    assert st == 1
    assert "device memory" in lib.xs_last_error().decode()
    big = nat.QGrid(0, 65537, 0, 1, 0, 1)
    st = lib.xs_intensity_fp32_static(ctypes.byref(tr), ctypes.byref(big), I.ctypes.data, None, None, None)
    assert st == 1 and "extent" in lib.xs_last_error().decode()
    many = nat.Traj(pos.ctypes.data, 0, f.ctypes.data, (1 << 31) + 1, 2, api._box(np.eye(3) * 10.0))
    st = lib.xs_intensity_fp32_static(ctypes.byref(many), ctypes.byref(g), I.ctypes.data, None, None, None)
    assert st == 1 and "2^31" in lib.xs_last_error().decode()
    assert lib.xs_intensity_fp32_static(None, ctypes.byref(g), I.ctypes.data, None, None, None) == 1


def test_batched_pipeline_rejects_missing_requests(lib):
    assert lib.xs_xpcs_batched(None, None, None, 1, 1, None, None, None) == 1
