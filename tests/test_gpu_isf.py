"""Intermediate scattering function and the contrast it predicts
(Sec. 2.3 Eqs. Fq_pq, norm_Fq, g2_from_fq, beta_alt_int) through the C ABI:
stage parity against the FP64 oracle on the same amplitudes, end to end on
the 4,000-atom workload (FP32 path, <= 1e-6) and on 256,000-atom frames (split
FP16 path, <= 1e-4), the AR(1) closed forms, the Siegert checks on a Brownian
ideal gas, and argument checks."""
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


def _c(amp):
    a = amp.detach().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("T,P,taus", [(1, 37, [0]), (10, 4096, list(range(10))),
                                      (200, 1000, [0, 1, 3, 64, 65, 199]), (129, 300, list(range(0, 129, 7)))])
def test_isf_stage_parity(xs, T, P, taus):
    g = torch.Generator().manual_seed(T * 1000 + P)
    amp = torch.randn((T, P, 2), generator=g).cuda()
    F, Fh = xs.isf(amp, taus, 3.5)
    xs.Context.get().sync_status()
    Fr, Fhr = oracle.isf(_c(amp.reshape(T, P, 2)), taus, 3.5)
    scale = (np.abs(_c(amp)) ** 2).mean(axis=0) / 3.5          # F(q, 0)
    assert np.all(np.abs(F.cpu().numpy() - Fr) <= 1e-6 * scale + 1e-12)
    assert np.all(np.abs(Fh.cpu().numpy() - Fhr) <= 1e-6)


def test_isf_config0_end_to_end_fp32(xs):
    traj, grid = wl.config0()
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    _, A = xs.intensity(p, fd, traj.box, grid, "fp32", want_amp=True)
    taus = list(range(10))
    sf2 = float((traj.f.astype(np.float64) ** 2).sum())
    F, Fh = xs.isf(A, taus, sf2)
    xs.Context.get().sync_status()
    m = grid.miller()
    Fr, Fhr = oracle.isf(oracle.amplitude(traj.pos, traj.f, traj.box, m), taus, sf2)
    nz = np.any(m != 0, axis=1)
    Fg = F.cpu().numpy()
    e_F = np.linalg.norm(Fg[:, nz] - Fr[:, nz]) / np.linalg.norm(Fr[:, nz])
    assert e_F <= 1e-6, e_F
    z = ~nz
    assert np.max(np.abs(Fg[:, z] - Fr[:, z]) / np.abs(Fr[:, z])) <= 1e-6


def test_isf_split_path_crystal_frames(xs):
    traj, grid = wl.config1(n_frames=48)
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    _, A = xs.intensity(p, fd, traj.box, grid, "fp16", want_amp=True)
    taus = [0, 1, 5, 47]
    sf2 = float((traj.f.astype(np.float64) ** 2).sum())
    F, Fh = xs.isf(A, taus, sf2)
    xs.Context.get().sync_status()
    m = grid.miller()
    rng = np.random.default_rng(5)
    pix = np.unique(np.concatenate([np.flatnonzero(np.all(m == 0, axis=1)), rng.choice(m.shape[0], 256, replace=False)]))
    Fr, Fhr = oracle.isf(oracle.amplitude(traj.pos, traj.f, traj.box, m[pix]), taus, sf2)
    Fg = F.cpu().numpy()[:, pix]
    nz = np.any(m[pix] != 0, axis=1)
    for k in range(len(taus)):
        e = np.linalg.norm(Fg[k, nz] - Fr[k, nz]) / np.linalg.norm(Fr[k, nz])
        assert e <= 1e-4, (taus[k], e)


def test_contrast_from_isf_stage_parity_and_ar1_closed_form(xs):
    # AR(1) amplitudes, rho set per ring; F_hat = rho^tau in expectation, the
    # contrast ratio follows from F_hat and matches the XSVS contrast of |a|^2
    T, Kmax = 3000, 40
    grid = wl.centered_plane(64)
    box = wl.cubic_box(50.0)
    m = grid.miller()
    n_rings = 20
    rings = oracle.ring_index(box, m, 1.0, n_rings)
    rho = (0.5 + 0.4 * rings / n_rings).astype(np.float32)
    A = wl.speckle_amplitudes(wl.SEED_BASE + 41, T, torch.from_numpy(rho), "cuda")
    _, Fh = xs.isf(A, list(range(Kmax)), 1.0)
    Ks = [1, 2, 7, 40, 10]
    ratio, counts = xs.contrast_from_isf(Fh, grid, box, Ks, n_rings)
    I = (A[..., 0] ** 2 + A[..., 1] ** 2).contiguous()
    beta, _ = xs.xsvs_contrast(I.view(T, 1, grid.ny, grid.nx), grid, box, Ks, n_rings)
    xs.Context.get().sync_status()
    ref, cref = oracle.contrast_from_isf(Fh.cpu().numpy(), Ks, rings, n_rings)
    assert np.array_equal(counts, cref)
    r = ratio.cpu().numpy()
    assert np.allclose(r, ref, rtol=1e-12, atol=0, equal_nan=True)
    b = beta.cpu().numpy()
    for ring in (5, 12, 19):
        x = float(rho[rings == ring][0]) ** 2
        for ik, K in enumerate(Ks):
            closed = (K * (1 + x) / (1 - x) - 2 * x * (1 - x ** K) / (1 - x) ** 2) / K ** 2
            assert abs(r[ik, ring - 1] - closed) < 0.03 * closed, (ring, K, r[ik, ring - 1], closed)
            if ring >= 12:   # enough pixels for the XSVS estimate (about 1/sqrt(n W) noise)
                xsvs = b[ik, ring - 1] / b[0, ring - 1]
                assert abs(xsvs - r[ik, ring - 1]) < 0.08 * closed, (ring, K, xsvs, r[ik, ring - 1])


def test_brownian_gas_siegert_relation(xs):
    # independent Brownian atoms (steps along x only): g2 - 1 = beta0 |F_hat|^2.
    # D q^2 >= 0.08 on every plane keeps the finite-T bias of the g2 estimate
    # (about 3 coth(D q^2) / T) below 0.01
    N, T, L, sig = 2000, 4000, 30.0, 2.0
    rng = np.random.default_rng(16)
    base = rng.random((N, 3)) * L
    steps = np.zeros((T, N, 3), dtype=np.float32)
    steps[1:, :, 0] = rng.standard_normal((T - 1, N)) * sig
    pos = (base[None] + np.cumsum(steps, axis=0, dtype=np.float64)).astype(np.float32)
    grid = wl.QGrid(1, 4, -8, 16, -8, 16)
    p = torch.from_numpy(pos).cuda()
    fd = torch.ones(N, device="cuda")
    I, A = xs.intensity(p, fd, np.eye(3) * L, grid, "fp16", want_amp=True)
    taus = [1, 2, 4]
    _, Fh = xs.isf(A, taus, float(N))
    g, _ = xs.g2(I.reshape(T, -1), taus)
    xs.Context.get().sync_status()
    m = grid.miller()
    Fh = Fh.cpu().numpy()
    g = g.cpu().numpy()
    beta0 = 1 - 1.0 / N
    D = sig * sig / 2
    for nx in range(1, 5):
        sel = m[:, 0] == nx
        q2 = (2 * math.pi * nx / L) ** 2
        for k, tau in enumerate(taus):
            want = math.exp(-D * q2 * tau)
            est = Fh[k, sel].real.mean()
            assert abs(est - want) < 5 * Fh[k, sel].real.std() / math.sqrt(sel.sum()) + 0.02, (nx, tau, est, want)
            lhs = (g[k, sel] - 1).mean() / beta0
            rhs = (np.abs(Fh[k, sel]) ** 2).mean()
            assert abs(lhs - rhs) < 5 * (g[k, sel] - 1).std() / math.sqrt(sel.sum()) + 0.02, (nx, tau, lhs, rhs)


def test_isf_argument_checks(xs):
    from paper_2204_13241_gb300._native import XsError
    amp = torch.zeros((4, 3, 2), device="cuda")
    with pytest.raises(XsError):
        xs.isf(amp, [4], 1.0)
    with pytest.raises(XsError):
        xs.isf(amp, [0], 0.0)
    Fh = torch.zeros((3, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(XsError):
        xs.contrast_from_isf(Fh, wl.centered_plane(4), np.eye(3), [4], 2)
    r, c = xs.contrast_from_isf(Fh, wl.centered_plane(4), np.eye(3), [], 2)
    assert r.shape == (0, 2)
