"""xs_intensity_fp32_static: the FP32 direct-sum intensity for callers that
cannot allocate device memory when they need it (hosts with a device memory
budget fixed at start-up, plug-ins inside an application that owns the
device memory, processes whose framework allocator already holds the
device).  Its scratch is a static device array, so it must give what
xs_intensity gives on the same inputs.  This file runs last: two calls in a
row through the C ABI, each compared with the context-based entry point at
the FP32 path's 1e-6, and the first also with the FP64 oracle; host buffers
are refused before any kernel runs."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_I, e_I
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import _native
    return _native.load()


def _case(seed, N, T, L):
    rng = np.random.default_rng(seed)
    base = rng.random((N, 3)) * L
    steps = rng.standard_normal((T, N, 3)) * 0.2
    steps[0] = 0
    pos = (base[None] + np.cumsum(steps, axis=0)).astype(np.float32)
    f = np.where(rng.random(N) < 0.5, 1.0, 0.6).astype(np.float32)
    return pos, f, np.eye(3) * L


def test_static_scratch_entry_matches_xs_intensity_on_two_calls(lib):
    from paper_2204_13241_gb300 import _native as nat
    from paper_2204_13241_gb300 import api

    cases = [(3000, 3, wl.QGrid(-32, 64, -32, 64, 0, 1), 25.0),
             (1234, 2, wl.QGrid(-20, 40, -9, 30, -1, 3), 17.0)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = []
    for i, (N, T, grid, L) in enumerate(cases):
        pos, f, box = _case(40 + i, N, T, L)
        p = torch.from_numpy(pos).cuda()
        fd = torch.from_numpy(f).cuda()
        shape = (T, grid.nz, grid.ny, grid.nx)
        I = torch.full(shape, -1.0, dtype=torch.float32, device="cuda")
        A = torch.full(shape + (2,), -1.0, dtype=torch.float32, device="cuda")
        tr = nat.Traj(p.data_ptr(), 0, fd.data_ptr(), N, T, api._box(box))
        g = nat.QGrid(*grid.as_tuple())
        st = lib.xs_intensity_fp32_static(ctypes.byref(tr), ctypes.byref(g), I.data_ptr(), A.data_ptr(),
                                          err.data_ptr(), stream)
        assert st == 0, lib.xs_last_error().decode()
        outs.append((p, fd, box, grid, I, A, pos, f))
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    # the first call against the FP64 oracle as well
    p, fd, box, grid, I, A, pos, f = outs[0]
    ref = oracle.intensity(pos, f, box, grid.miller())
    check_I(I.reshape(I.shape[0], -1).cpu().numpy(), ref, grid.miller(), "fp32")
    for p, fd, box, grid, I, A, _, _ in outs:
        I_ref, A_ref = api.intensity(p, fd, box, grid, "fp32", want_amp=True)
        api.Context.get().sync_status()
        m = grid.miller()
        ref = I_ref.reshape(I_ref.shape[0], -1).cpu().numpy().astype(np.float64)
        got = I.reshape(I.shape[0], -1).cpu().numpy()
        e, e0 = e_I(got, ref, m)
        assert e <= 1e-6 and e0 <= 1e-6, (e, e0)
        a = A.cpu().numpy().astype(np.float64)
        a_ref = A_ref.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - a_ref) <= 1e-6 * np.linalg.norm(a_ref)


def test_static_scratch_entry_rejects_oversized_requests(lib):
    from paper_2204_13241_gb300 import _native as nat
    from paper_2204_13241_gb300 import api

    # 400 frames x 100,000 atoms of phase records alone need 640 MB
    p = torch.empty((400, 100_000, 3), dtype=torch.float32, device="cuda")
    fd = torch.ones(100_000, dtype=torch.float32, device="cuda")
    I = torch.empty((400, 1, 8, 8), dtype=torch.float32, device="cuda")
    tr = nat.Traj(p.data_ptr(), 0, fd.data_ptr(), 100_000, 400, api._box(np.eye(3) * 50.0))
    g = nat.QGrid(-4, 8, -4, 8, 0, 1)
    st = lib.xs_intensity_fp32_static(ctypes.byref(tr), ctypes.byref(g), I.data_ptr(), None, None,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    assert "static scratch holds" in lib.xs_last_error().decode()


def test_static_scratch_entry_refuses_host_buffers(lib):
    from paper_2204_13241_gb300 import _native as nat
    from paper_2204_13241_gb300 import api

    p = torch.zeros((1, 16, 3), dtype=torch.float32, device="cuda")
    fd = torch.ones(16, dtype=torch.float32, device="cuda")
    I_host = torch.zeros((1, 1, 8, 8), dtype=torch.float32)
    tr = nat.Traj(p.data_ptr(), 0, fd.data_ptr(), 16, 1, api._box(np.eye(3) * 10.0))
    g = nat.QGrid(-4, 8, -4, 8, 0, 1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.xs_intensity_fp32_static(ctypes.byref(tr), ctypes.byref(g), I_host.data_ptr(), None, None, stream)
    assert st == 1 and "device memory" in lib.xs_last_error().decode()
    pos_host = torch.zeros((1, 16, 3), dtype=torch.float32)
    tr = nat.Traj(pos_host.data_ptr(), 0, fd.data_ptr(), 16, 1, api._box(np.eye(3) * 10.0))
    I = torch.zeros((1, 1, 8, 8), dtype=torch.float32, device="cuda")
    st = lib.xs_intensity_fp32_static(ctypes.byref(tr), ctypes.byref(g), I.data_ptr(), None, None, stream)
    assert st == 1 and "device memory" in lib.xs_last_error().decode()
