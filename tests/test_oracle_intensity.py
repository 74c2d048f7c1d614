"""Pins of the FP64 oracle's intensity against closed forms, invariants and
brute force (arXiv 2204.13241 Sec. 2.1-2.2 and Sec. 3.1).

None of these tests retypes the oracle's own formula: each compares it with
a different statement of the physics (pair sum, crystal selection rules,
two-atom interference, periodic images, statistics of an ideal gas)."""
import math

import numpy as np
import pytest

import oracle
from paper_2204_13241_gb300 import workloads as wl


def _rng(k):
    return np.random.default_rng(1000 + k)


def _cubic(L):
    return np.eye(3) * L


def test_forward_scattering_is_total_form_factor_squared():
    # |S(0)|^2 = (sum f)^2 for any configuration
    rng = _rng(1)
    pos = (rng.random((3, 300, 3)) * 25).astype(np.float32)
    f = rng.uniform(0.2, 2.0, 300)
    I = oracle.intensity(pos, f, _cubic(25.0), np.array([[0, 0, 0]]))
    assert np.allclose(I[:, 0], f.sum() ** 2, rtol=1e-13)


def test_single_atom_gives_f_squared_and_phase_sign():
    rng = _rng(2)
    r = np.array([[3.25, -7.5, 11.125]], dtype=np.float32)
    L = 17.0
    g = wl.QGrid(-4, 9, -3, 7, -2, 5)
    m = g.miller()
    S = oracle.amplitude(r, np.array([1.7]), _cubic(L), m)[0]
    assert np.allclose(np.abs(S) ** 2, 1.7 ** 2, rtol=1e-13)
    # sign convention: S = f exp(+i q.r) with q = 2 pi n / L
    th = 2 * math.pi * (m.astype(np.float64) @ r[0].astype(np.float64)) / L
    assert np.allclose(S, 1.7 * np.exp(1j * th), atol=1e-12)


def test_two_atoms_interference():
    # I = f1^2 + f2^2 + 2 f1 f2 cos(q.(r1 - r2))   (Eq. Iq_rij with N = 2)
    r = np.array([[1.5, 2.25, -0.75], [9.0, -4.5, 6.0]], dtype=np.float32)
    f = np.array([1.3, 0.4])
    L = 13.0
    m = wl.QGrid(-5, 11, -5, 11, 2, 1).miller()
    I = oracle.intensity(r, f, _cubic(L), m)[0]
    dr = (r[0].astype(np.float64) - r[1].astype(np.float64))
    ref = f[0] ** 2 + f[1] ** 2 + 2 * f[0] * f[1] * np.cos(2 * math.pi * (m @ dr) / L)
    assert np.allclose(I, ref, rtol=1e-12, atol=1e-12)


def _pair_sum(pos, f, q):
    # brute-force Eq. Iq_rij: sum_i sum_j f_i f_j exp(-i q.(r_i - r_j))
    d = pos[:, None, :] - pos[None, :, :]                  # [N][N][3]
    ph = np.einsum("ijk,pk->pij", d, q)                    # [P][N][N]
    return np.real((f[None, :, None] * f[None, None, :] * np.exp(-1j * ph)).sum(axis=(1, 2)))


def test_pair_sum_equals_single_sum_bruteforce():
    rng = _rng(3)
    for N in (1, 2, 7, 33, 64):
        pos = (rng.random((N, 3)) * 11).astype(np.float32)
        f = rng.uniform(0.1, 1.5, N)
        L = 11.0
        m = wl.QGrid(-3, 7, -2, 5, -1, 3).miller()
        q = 2 * math.pi * m.astype(np.float64) / L
        ref = _pair_sum(pos.astype(np.float64), f, q)
        I = oracle.intensity(pos, f, _cubic(L), m)[0]
        assert np.allclose(I, ref, rtol=1e-11, atol=1e-9 * f.sum() ** 2)


def test_translation_and_periodic_images_do_not_change_intensity():
    rng = _rng(4)
    N, L = 120, 19.0
    # positions on a 2^-10 grid so that the shifts below are exact in float32
    pos = (np.round(rng.random((N, 3)) * L * 1024) / 1024).astype(np.float32)
    f = rng.uniform(0.5, 1.5, N)
    m = wl.QGrid(-6, 12, -6, 12, 1, 1).miller()
    I0 = oracle.intensity(pos, f, _cubic(L), m)[0]
    shifted = (pos + np.array([3.0, -5.5, 7.25], dtype=np.float32)).astype(np.float32)
    I1 = oracle.intensity(shifted, f, _cubic(L), m)[0]
    assert np.allclose(I1, I0, rtol=1e-9, atol=1e-9 * N)
    images = pos + (rng.integers(-3, 4, (N, 3)) * L).astype(np.float32)
    I2 = oracle.intensity(images.astype(np.float32), f, _cubic(L), m)[0]
    assert np.allclose(I2, I0, rtol=1e-9, atol=1e-9 * N)


def test_triclinic_cell_lattice_vectors_are_periods():
    # With h's columns as the cell edges, r -> r + h m (integer m) is a period of
    # exp(i q.r) for q = 2 pi h^-T n.  A transposed h would fail this.
    rng = _rng(5)
    h = np.array([[12.0, 3.0, -1.5], [0.0, 10.0, 2.5], [1.0, 0.0, 9.0]])
    N = 60
    s = rng.random((N, 3))
    pos = (s @ h.T).astype(np.float32)
    f = rng.uniform(0.5, 1.5, N)
    m = wl.QGrid(-3, 7, -3, 7, -2, 5).miller()
    S0 = oracle.amplitude(pos, f, h, m)[0]
    shift = rng.integers(-2, 3, (N, 3)).astype(np.float64)
    pos2 = (pos.astype(np.float64) + shift @ h.T)
    S1 = oracle.amplitude(pos2.astype(np.float32), f, h, m)[0]
    assert np.allclose(S1, S0, atol=2e-4 * N)
    # and the same holds for whole-crystal translation on intensities only
    q = oracle.qvectors(h, m)
    assert np.allclose(q @ h, 2 * math.pi * m, atol=1e-10)


def test_friedel_symmetry():
    rng = _rng(6)
    pos = (rng.random((1, 200, 3)) * 30).astype(np.float32)
    f = rng.uniform(0.3, 1.0, 200)
    m = wl.QGrid(-5, 11, -5, 11, -1, 3).miller()
    I = oracle.intensity(pos, f, _cubic(30.0), m)[0]
    I_neg = oracle.intensity(pos, f, _cubic(30.0), -m)[0]
    assert np.allclose(I, I_neg, rtol=1e-12, atol=1e-10)


def test_perfect_fcc_selection_rules():
    cells, a = 3, 4.0
    sites = wl.fcc_sites(cells, a).astype(np.float32)
    N = sites.shape[0]
    L = cells * a
    m = wl.QGrid(-7, 15, -7, 15, -3, 7).miller()
    I = oracle.intensity(sites, np.ones(N), _cubic(L), m)[0]
    hkl = m // cells
    on_lattice = np.all(m % cells == 0, axis=1)
    par = hkl % 2
    same_parity = np.all(par == par[:, :1], axis=1)
    allowed = on_lattice & same_parity
    assert allowed.sum() > 5 and (~allowed).sum() > 100
    assert np.allclose(I[allowed], N * N, rtol=1e-10)
    assert np.all(I[~allowed] <= 1e-12 * N * N)


def test_ideal_gas_mean_intensity_is_sum_f_squared():
    # independent uniform atoms: <I(q)> = sum f^2 for every q != 0 on the lattice,
    # and I is exponentially distributed (Sec. 4.3), so the std of I is ~ <I>.
    rng = _rng(7)
    N, L, T = 400, 20.0, 6
    pos = (rng.random((T, N, 3)) * L).astype(np.float32)
    f = np.where(rng.random(N) < 0.5, 1.0, 0.6)
    m = wl.QGrid(-8, 16, -8, 16, 0, 1).miller()
    m = m[np.any(m != 0, axis=1)]
    I = oracle.intensity(pos, f, _cubic(L), m)
    s2 = (f ** 2).sum()
    n = I.size
    assert abs(I.mean() - s2) < 5 * s2 / math.sqrt(n)
    # exponential statistics: contrast <I^2>/<I>^2 - 1 near 1
    beta = (I ** 2).mean() / I.mean() ** 2 - 1
    assert abs(beta - 1.0) < 0.1
