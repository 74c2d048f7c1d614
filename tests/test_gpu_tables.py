"""The two table builders of the tensor-core path on the 256,000-atom /
1,000-frame / 128^2 workload at full size (Sec. 3.1: each table entry is
exp(i 2 pi n s) of an atom's fractional coordinate).  The default builder
evaluates a seed and a step per run in FP32 and advances by complex
multiplication; the FP64 builder evaluates every entry with sincospi of its
exact turn count.  Both must meet the split path's bounds against the FP64
oracle, and they must agree with each other to within the contraction's own
rounding, which shows that the recurrence adds no error of its own."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_I, e_I, e_pix
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


def test_fp64_and_recurrence_builders_on_the_full_workload(xs):
    traj, grid = wl.config1()
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    ctx = xs.Context.get()
    I_rec = xs.intensity(p, fd, traj.box, grid, "fp16")
    ctx.sync_status()
    ctx.set_table_builder(True)
    try:
        I_ex = xs.intensity(p, fd, traj.box, grid, "fp16")
        ctx.sync_status()
    finally:
        ctx.set_table_builder(False)
    del p
    m = grid.miller()
    frames = [0, 500, 999]
    rng = np.random.default_rng(98)
    pix = np.unique(np.concatenate([[np.flatnonzero(np.all(m == 0, axis=1))[0]],
                                    rng.choice(m.shape[0], 1024, replace=False)]))
    ref = oracle.intensity(traj.pos[frames], traj.f, traj.box, m[pix])
    a = I_rec.reshape(1000, -1)[frames][:, pix].cpu().numpy()
    b = I_ex.reshape(1000, -1)[frames][:, pix].cpu().numpy()
    check_I(a, ref, m[pix], "fp16", what="recurrence builder")
    check_I(b, ref, m[pix], "fp16", what="FP64 builder")
    # the builders differ only in the last bits of the table entries: whole
    # series, every pixel
    A = I_rec.reshape(1000, -1).cpu().numpy()
    B = I_ex.reshape(1000, -1).cpu().numpy().astype(np.float64)
    assert e_I(A, B, m)[0] <= 1e-4
    assert e_pix(A, B, m) <= 2e-3


def test_fp64_builder_on_both_tile_kinds_and_a_volume(xs):
    rng = np.random.default_rng(12)
    N, T, L = 5000, 2, 31.0
    pos = (rng.random((T, N, 3)) * L).astype(np.float32)
    f = rng.uniform(0.5, 1.5, N).astype(np.float32)
    box = np.eye(3) * L
    ctx = xs.Context.get()
    p, fd = torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda()
    for grid in (wl.centered_plane(64), wl.QGrid(-20, 150, -70, 140, 2, 1), wl.QGrid(-9, 19, -9, 19, -9, 19)):
        ctx.set_table_builder(True)
        try:
            I = xs.intensity(p, fd, box, grid, "bf16")
            ctx.sync_status()
        finally:
            ctx.set_table_builder(False)
        m = grid.miller()
        check_I(I.reshape(T, -1).cpu().numpy(), oracle.intensity(pos, f, box, m), m, "bf16", what=str(grid))
