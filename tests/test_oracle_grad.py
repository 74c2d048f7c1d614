"""Pins of the oracle's position gradient: FP64 central finite differences
(an independent evaluation through the loss), torch float64 autograd of a
plain direct-sum loss, translation invariance and the q_z = 0 plane."""
import math

import numpy as np
import pytest

import oracle
from paper_2204_13241_gb300 import workloads as wl


def _case(seed=5, N=40, L=14.0, side=8):
    rng = np.random.default_rng(seed)
    pos = (rng.random((N, 3)) * L).astype(np.float32)
    target = (pos + rng.standard_normal(pos.shape) * 0.3).astype(np.float32)
    f = rng.uniform(0.5, 1.5, N)
    grid = wl.centered_plane(side, nz=0)
    m = grid.miller()
    box = np.eye(3) * L
    w = 1.0 / (1.0 + ((2 * math.pi * m / L) ** 2).sum(axis=1))
    It = oracle.intensity(target, f, box, m)[0]
    return pos, f, box, m, w, It


def test_analytic_gradient_matches_central_differences():
    pos, f, box, m, w, It = _case()
    I = oracle.intensity(pos, f, box, m)[0]
    G = 2 * w * (I - It)
    g = oracle.grad_analytic(pos, f, box, m, G)
    atoms = list(range(0, pos.shape[0], 3))
    g_fd = oracle.grad_fd(pos, f, box, m, lambda I1: (w * (I1 - It) ** 2).sum(), atoms, h=1e-4)
    err = np.linalg.norm(g[atoms] - g_fd) / np.linalg.norm(g_fd)
    assert err < 1e-6


def test_gradient_sums_to_zero_and_vanishes_along_z_on_qz0_plane():
    pos, f, box, m, w, It = _case(seed=9)
    I = oracle.intensity(pos, f, box, m)[0]
    G = 2 * w * (I - It)
    g = oracle.grad_analytic(pos, f, box, m, G)
    scale = np.abs(g).max()
    assert np.all(np.abs(g.sum(axis=0)) < 1e-9 * scale * pos.shape[0])
    assert np.all(np.abs(g[:, 2]) < 1e-12 * scale)


def test_gradient_matches_torch_autograd_of_direct_sum():
    torch = pytest.importorskip("torch")
    pos, f, box, m, w, It = _case(seed=13, N=25, side=6)
    m3 = wl.QGrid(-3, 6, -3, 6, -1, 3).miller()     # a volume, so z is exercised
    L = box[0, 0]
    w3 = 1.0 / (1.0 + ((2 * math.pi * m3 / L) ** 2).sum(axis=1))
    It3 = np.random.default_rng(2).random(m3.shape[0]) * 30
    r = torch.tensor(pos.astype(np.float64), requires_grad=True)
    q = torch.tensor(2 * math.pi * m3.astype(np.float64) / L)
    th = r @ q.T                                               # [N][P]
    ft = torch.tensor(f)[:, None]
    re = (ft * torch.cos(th)).sum(0)
    im = (ft * torch.sin(th)).sum(0)
    I = re * re + im * im
    loss = (torch.tensor(w3) * (I - torch.tensor(It3)) ** 2).sum()
    loss.backward()
    I_or = oracle.intensity(pos, f, box, m3)[0]
    G = 2 * w3 * (I_or - It3)
    g = oracle.grad_analytic(pos, f, box, m3, G)
    ref = r.grad.numpy()
    assert np.allclose(g, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
