"""The FFT-based method (Sec. 3.2, Algorithm 2) through xs_intensity_fft, a
cross-check of the direct method: parity with the FP64 oracle's Algorithm 2
on the same grid, agreement with the direct sum where the grid resolves q,
the one-atom closed form, and argument checks."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import e_I, e_pix
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


def _gas(seed, N, T, L):
    rng = np.random.default_rng(seed)
    pos = (rng.random((T, N, 3)) * np.array(L)).astype(np.float32)
    f = (rng.random(N) + 0.5).astype(np.float32)
    return pos, f, np.diag(np.array(L, dtype=np.float64))


def test_fft_method_matches_oracle_algorithm_2_and_direct_sum(xs):
    pos, f, box = _gas(1, 300, 3, (12.0, 12.0, 12.0))
    grid = wl.QGrid(-8, 16, -8, 16, -3, 7)
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    I = xs.intensity_fft(p, fd, box, grid, 64, 0.35)
    xs.Context.get().sync_status()
    m = grid.miller()
    got = I.reshape(I.shape[0], -1).cpu().numpy()
    alg2 = oracle.fft_intensity(pos, f, box, 64, 0.35, 0, m)
    e, e0 = e_I(got, alg2, m)
    assert e <= 1e-6 and e0 <= 1e-6, (e, e0)             # same method, FP64 on both sides
    assert e_pix(got, alg2, m) <= 5e-6                   # float32 output of an FP64 result
    direct = oracle.intensity(pos, f, box, m)
    e, e0 = e_I(got, direct, m)
    assert e <= 1e-4 and e0 <= 1e-4, (e, e0)             # the method's own grid and cut-off error
    assert e_pix(got, direct, m) <= 2e-3


def test_fft_method_orthorhombic_plane_and_one_atom(xs):
    pos, f, box = _gas(2, 500, 2, (16.0, 12.0, 20.0))
    grid = wl.centered_plane(32, nz=2)
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    I = xs.intensity_fft(p, fd, box, grid, 128, 0.3)
    xs.Context.get().sync_status()
    m = grid.miller()
    alg2 = oracle.fft_intensity(pos, f, box, 128, 0.3, 0, m)
    e, _ = e_I(I.reshape(2, -1).cpu().numpy(), alg2, m)
    assert e <= 1e-6, e
    assert e_pix(I.reshape(2, -1).cpu().numpy(), alg2, m) <= 5e-6
    # one atom on a grid point: I = f^2 at every q
    h = 16.0 / 128
    one = torch.tensor([[[5 * h, 0.0, 0.0]]], device="cuda")
    I1 = xs.intensity_fft(one, torch.tensor([1.3], device="cuda"), box, grid, 128, 0.3)
    xs.Context.get().sync_status()
    assert torch.allclose(I1, torch.full_like(I1, 1.69), rtol=1e-6, atol=0)   # float32 output


def test_fft_method_argument_checks(xs):
    from paper_2204_13241_gb300._native import XsError
    pos, f, box = _gas(3, 10, 1, (10.0, 10.0, 10.0))
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    tri = box.copy()
    tri[0, 1] = 1.0
    with pytest.raises(XsError):
        xs.intensity_fft(p, fd, tri, wl.centered_plane(8), 32, 0.3)
    with pytest.raises(XsError):
        xs.intensity_fft(p, fd, box, wl.centered_plane(8), 48, 0.3)     # not a power of two
    with pytest.raises(XsError):
        xs.intensity_fft(p, fd, box, wl.centered_plane(64), 32, 0.3)    # outside [-16, 16)
