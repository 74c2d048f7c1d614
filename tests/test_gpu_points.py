"""Intensity at arbitrary reciprocal-lattice points and on the Ewald-sphere
detector slice (Fig. 5, |k_f| = |k_i|) through xs_intensity_points: parity
with the FP64 oracle on the FP32 direct path (<= 1e-6) and the tensor-core
path (points grouped by n_z plane, <= 1e-4), agreement with xs_intensity when
the points are a whole plane, and edge cases."""
import math

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


def test_ewald_slice_fp32_4000_atoms(xs):
    traj, _ = wl.config0()
    m, valid = xs.ewald_points(traj.box, [0.0, 0.0, 2 * math.pi / 1.5], -32, 64, -32, 64)
    pts = m[valid]
    assert len(np.unique(pts[:, 2])) > 10          # a curved slice: many n_z planes
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I, A = xs.intensity_points(p, fd, traj.box, pts, "fp32", want_amp=True)
    xs.Context.get().sync_status()
    S = oracle.amplitude(traj.pos, traj.f, traj.box, pts)
    ref = S.real ** 2 + S.imag ** 2
    check_I(I.cpu().numpy(), ref, pts, "fp32")
    a = A.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a[..., 0] + 1j * a[..., 1] - S) <= 1e-6 * np.linalg.norm(S)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_ewald_slice_split_path_crystal(xs, prec):
    traj, _ = wl.config1(n_frames=4)
    m, valid = xs.ewald_points(traj.box, [0.0, 0.0, 2 * math.pi / 0.9], -150, 300, -140, 280)
    pts = m[valid]
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I = xs.intensity_points(p, fd, traj.box, pts, prec)
    xs.Context.get().sync_status()
    rng = np.random.default_rng(9)
    sel = np.unique(np.concatenate([np.flatnonzero(np.all(pts == 0, axis=1)), rng.choice(len(pts), 512, replace=False)]))
    ref = oracle.intensity(traj.pos[[0, 3]], traj.f, traj.box, pts[sel])
    check_I(I.cpu().numpy()[[0, 3]][:, sel], ref, pts[sel], prec)


def test_points_of_a_whole_plane_equal_the_plane(xs):
    traj, grid = wl.config0(keep=[0, 4, 9])
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    m = grid.miller()
    for prec, tol in (("fp32", 1e-6), ("fp16", 1e-5)):
        Ip = xs.intensity_points(p, fd, traj.box, m, prec)
        Ig = xs.intensity(p, fd, traj.box, grid, prec)
        xs.Context.get().sync_status()
        Ig64 = Ig.reshape(Ig.shape[0], -1).cpu().numpy().astype(np.float64)
        e, _ = e_I(Ip.cpu().numpy(), Ig64, m)
        assert e <= tol, (prec, e)
        assert e_pix(Ip.cpu().numpy(), Ig64, m) <= 10 * tol, prec


def test_points_edge_cases(xs):
    from paper_2204_13241_gb300._native import XsError
    traj, _ = wl.config0(keep=[0])
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    # one point, far from the origin, on its own plane; q = 0 gives (sum f)^2
    pts = np.array([[0, 0, 0], [97, -45, 61]], dtype=np.int32)
    for prec in ("fp32", "fp16"):
        I = xs.intensity_points(p, fd, traj.box, pts, prec)
        xs.Context.get().sync_status()
        ref = oracle.intensity(traj.pos, traj.f, traj.box, pts)
        assert abs(I[0, 0].item() - ref[0, 0]) <= 1e-6 * ref[0, 0]
        assert abs(I[0, 1].item() - ref[0, 1]) <= 1e-4 * ref[0, 0] / 4000
    empty = xs.intensity_points(p, fd, traj.box, np.zeros((0, 3), np.int32), "fp16")
    assert empty.shape == (1, 0)
    with pytest.raises(ValueError):
        xs.intensity_points(p.cpu(), fd.cpu(), traj.box, pts, "fp16")
