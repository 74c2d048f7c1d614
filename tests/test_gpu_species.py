"""Several atom species with q-dependent form factors (Sec. 2.1, f_i(q) as a
sum of Gaussians per species) through xs_intensity_species: parity against the
FP64 oracle on the FP32 path (<= 1e-6) and the split paths (<= 1e-4), the
single-constant-species reduction to xs_intensity, tracer labelling (Sec. 4.5:
only a labelled subset scatters) and argument checks."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_I
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# three synthetic species (a1, b1, .., a4, b4, c); b in A^2
COEF = np.array([[8.0, 12.0, 6.0, 1.5, 3.0, 40.0, 1.0, 0.3, 0.2],
                 [2.5, 6.0, 1.5, 0.8, 0.0, 1.0, 0.0, 1.0, 0.1],
                 [1.0, 20.0, 0.5, 2.0, 0.2, 60.0, 0.1, 0.5, 0.0]])


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


def _species(n, seed):
    return np.random.default_rng(seed).integers(0, 3, n).astype(np.int32)


def test_species_fp32_path_4000_atoms(xs):
    traj, grid = wl.config0()
    sp = _species(traj.n_atoms, 1)
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I, A = xs.intensity_species(p, fd, sp, COEF, traj.box, grid, "fp32", want_amp=True)
    xs.Context.get().sync_status()
    m = grid.miller()
    S = oracle.amplitude_species(traj.pos, traj.f, sp, COEF, traj.box, m)
    ref = S.real ** 2 + S.imag ** 2
    check_I(I.reshape(I.shape[0], -1).cpu().numpy(), ref, m, "fp32")
    a = A.reshape(A.shape[0], -1, 2).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a[..., 0] + 1j * a[..., 1] - S) <= 1e-6 * np.linalg.norm(S)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_species_split_path_crystal_frames(xs, prec):
    traj, grid = wl.config1(n_frames=6)
    sp = _species(traj.n_atoms, 2)
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I = xs.intensity_species(p, fd, sp, COEF, traj.box, grid, prec)
    xs.Context.get().sync_status()
    m = grid.miller()
    rng = np.random.default_rng(3)
    pix = np.unique(np.concatenate([np.flatnonzero(np.all(m == 0, axis=1)), rng.choice(m.shape[0], 512, replace=False)]))
    ref = oracle.intensity_species(traj.pos[[0, 5]], traj.f, sp, COEF, traj.box, m[pix])
    got = I.reshape(I.shape[0], -1)[[0, 5]][:, pix].cpu().numpy()
    check_I(got, ref, m[pix], prec)


def test_single_constant_species_equals_xs_intensity(xs):
    traj, grid = wl.config0(keep=[0, 1, 2])
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    one = np.array([[0, 0, 0, 0, 0, 0, 0, 0, 1.0]])
    for prec in ("fp32", "fp16"):
        a = xs.intensity_species(p, fd, np.zeros(traj.n_atoms, np.int32), one, traj.box, grid, prec)
        b = xs.intensity(p, fd, traj.box, grid, prec)
        xs.Context.get().sync_status()
        # the species path squares the FP32-rounded amplitude: about 1e-7 apart
        assert torch.allclose(a, b, rtol=1e-6, atol=0), prec


def test_tracer_labelling(xs):
    # 45 labelled atoms scatter, the other 3,955 do not: the same as the
    # labelled atoms alone
    traj, grid = wl.config0(keep=[0, 9])
    sp = np.zeros(traj.n_atoms, np.int32)
    sp[::89] = 1
    coef = np.array([[0, 0, 0, 0, 0, 0, 0, 0, 0.0], [0, 0, 0, 0, 0, 0, 0, 0, 1.0]])
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I = xs.intensity_species(p, fd, sp, coef, traj.box, grid, "fp32")
    sub = torch.from_numpy(np.ascontiguousarray(traj.pos[:, sp == 1])).cuda()
    J = xs.intensity(sub, fd[torch.from_numpy(sp == 1).cuda()].contiguous(), traj.box, grid, "fp32")
    xs.Context.get().sync_status()
    assert torch.allclose(I, J, rtol=1e-6, atol=1e-5)


def test_species_argument_checks(xs):
    from paper_2204_13241_gb300._native import XsError
    p = torch.zeros((1, 4, 3), device="cuda")
    fd = torch.ones(4, device="cuda")
    with pytest.raises(XsError):
        xs.intensity_species(p, fd, [0, 1, 2, 0], COEF[:2], np.eye(3) * 5, wl.centered_plane(8), "fp32")
    bad = COEF.copy()
    bad[0, 3] = np.nan
    with pytest.raises(XsError):
        xs.intensity_species(p, fd, [0, 1, 2, 0], bad, np.eye(3) * 5, wl.centered_plane(8), "fp32")
