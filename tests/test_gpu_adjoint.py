"""Parity of the CUDA adjoint dL/dr with the oracle's analytic gradient and
with FP64 central finite differences (h = 1e-4 A) of a caller loss
L = sum_q w_q (I_q - I_target,q)^2, w_q = 1/(1+|q|^2); relative L2 error
<= 1e-4 over the sampled components."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


def _weights(grid, L):
    m = grid.miller().astype(np.float64) * 2 * math.pi / L
    return 1.0 / (1.0 + (m ** 2).sum(axis=1))


@pytest.mark.parametrize("N,grid", [
    (300, wl.QGrid(-16, 32, -16, 32, 0, 1)),
    (1000, wl.QGrid(-20, 40, -9, 300, 0, 1)),     # n_y longer than one shared-memory chunk
    (129, wl.QGrid(-4, 9, -5, 11, -3, 7)),         # volume: z gradient non-zero
])
def test_adjoint_matches_oracle_gradient(xs, N, grid):
    rng = np.random.default_rng(N)
    L = 18.0
    pos = (rng.random((N, 3)) * L).astype(np.float32)
    f = rng.uniform(0.5, 1.5, N).astype(np.float32)
    G = rng.standard_normal(grid.n_pixels)
    amp = oracle.amplitude(pos, f, np.eye(3) * L, grid.miller())[0]
    A = np.stack([amp.real, amp.imag], axis=-1).astype(np.float32)
    g = xs.intensity_backward(torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda(), np.eye(3) * L, grid,
                              torch.from_numpy(A).cuda(), torch.from_numpy(G.astype(np.float32)).cuda())
    xs.Context.get().sync_status()
    ref = oracle.grad_analytic(pos, f, np.eye(3) * L, grid.miller(), G.astype(np.float32).astype(np.float64),
                               amp=A[..., 0].astype(np.float64) + 1j * A[..., 1].astype(np.float64))
    got = g.cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-4, err
    if grid.nz == 1 and grid.nz0 == 0:
        assert np.all(got[:, 2] == 0.0)


def test_autograd_function_chain_and_translation_invariance(xs):
    rng = np.random.default_rng(3)
    N, L = 500, 15.0
    grid = wl.QGrid(-12, 24, -12, 24, 0, 1)
    pos = torch.from_numpy((rng.random((N, 3)) * L).astype(np.float32)).cuda().requires_grad_(True)
    f = torch.ones(N, device="cuda")
    target = torch.from_numpy(rng.exponential(float(N), grid.n_pixels).astype(np.float32)).cuda()
    w = torch.from_numpy(_weights(grid, L).astype(np.float32)).cuda()
    I = xs.IntensityFn.apply(pos, f, np.eye(3) * L, grid)   # default: the factorised FP32 forward
    loss = (w * (I - target) ** 2).sum()
    loss.backward()
    g = pos.grad.detach().cpu().numpy()
    scale = np.abs(g).max()
    assert np.all(np.abs(g.sum(axis=0)) <= 1e-3 * scale * math.sqrt(N))
    # compare with the oracle through the same caller loss
    P = pos.detach().cpu().numpy()
    Iref = oracle.intensity(P, np.ones(N), np.eye(3) * L, grid.miller())[0]
    Gref = 2 * _weights(grid, L) * (Iref - target.cpu().numpy())
    ref = oracle.grad_analytic(P, np.ones(N), np.eye(3) * L, grid.miller(), Gref)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 1e-4


@pytest.mark.parametrize("prec", ["fp32", "fp32f"])
def test_config3_full_size_against_finite_differences(xs, prec):
    """100,000 atoms, 256^2 plane; 64 random atoms checked against FP64
    central differences of the loss (exact incremental S updates), with the
    forward (I and S) from the plain FP32 kernel or the factorised one."""
    traj, target, grid = wl.config3()
    L = traj.L
    m = grid.miller()
    w = _weights(grid, L)
    pos = torch.from_numpy(traj.pos[0]).cuda()
    f = torch.from_numpy(traj.f).cuda()
    It = oracle.intensity(target[0], traj.f, traj.box, m)[0]
    I, amp = xs.intensity(pos, f, traj.box, grid, prec, want_amp=True)
    G = 2 * torch.from_numpy(w.astype(np.float32)).cuda() * (I.reshape(-1) - torch.from_numpy(It.astype(np.float32)).cuda())
    g = xs.intensity_backward(pos, f, traj.box, grid, amp.reshape(-1, 2).contiguous(), G.contiguous())
    xs.Context.get().sync_status()
    atoms = np.random.default_rng(64).choice(traj.n_atoms, 64, replace=False)
    S = oracle.amplitude(traj.pos[0], traj.f, traj.box, m)[0]
    fd = oracle.grad_fd(traj.pos[0], traj.f, traj.box, m, lambda I1: float((w * (I1 - It) ** 2).sum()),
                        atoms, h=1e-4, amp=S)
    got = g.cpu().numpy()[atoms]
    err = np.linalg.norm(got - fd) / np.linalg.norm(fd)
    assert err <= 1e-4, err
