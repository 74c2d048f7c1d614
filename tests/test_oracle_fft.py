"""Pins of the oracle's FFT-based method (arXiv 2204.13241 Sec. 3.2,
Algorithm 2):
  * one atom on a grid point: its smeared density is the origin Gaussian
    shifted by whole grid steps, so I = f^2 exactly at every q;
  * convergence to the direct sum (Algorithm 1) on a well-resolved grid, and a
    larger error on a coarser grid and with a tight cut-off (the grid and
    truncation errors the paper discusses);
  * an orthorhombic cell is accepted, a triclinic one is refused."""
import numpy as np
import pytest

import oracle


def _case(seed, L=(12.0, 12.0, 12.0), N=40, T=2):
    rng = np.random.default_rng(seed)
    pos = (rng.random((T, N, 3)) * np.array(L)).astype(np.float32)
    f = rng.random(N) + 0.5
    m = np.array([[a, b, c] for a in range(-6, 7, 3) for b in range(-6, 7, 2) for c in (-4, 0, 5)])
    return pos, f, np.diag(L), m


def test_single_atom_on_a_grid_point_gives_f_squared():
    L, n = 12.0, 64
    h = L / n
    pos = np.array([[[15 * h, 0.0, 32 * h]]], dtype=np.float32)
    _, _, box, m = _case(0)
    I = oracle.fft_intensity(pos, [1.7], np.eye(3) * L, n, 0.35, 20, m)
    assert np.allclose(I, 1.7 ** 2, rtol=1e-12, atol=0)


def test_converges_to_the_direct_sum_and_degrades_as_expected():
    pos, f, box, m = _case(1)
    ref = oracle.intensity(pos, f, box, m)

    def err(n, eta, k):
        I = oracle.fft_intensity(pos, f, box, n, eta, k, m)
        return np.linalg.norm(I - ref) / np.linalg.norm(ref)

    fine = err(64, 0.35, 20)          # eta = 1.9 grid steps, cut-off +-5.4 eta
    assert fine < 1e-5, fine
    coarse = err(32, 0.35, 10)        # eta = 0.9 grid steps: aliasing
    tight = err(64, 0.35, 4)          # cut-off +-1.1 eta: truncation
    assert coarse > 10 * fine and tight > 10 * fine, (fine, coarse, tight)


def test_orthorhombic_cell_and_triclinic_refusal():
    pos, f, box, m = _case(2, L=(12.0, 9.0, 15.0))
    ref = oracle.intensity(pos, f, box, m)
    I = oracle.fft_intensity(pos, f, box, 96, 0.3, 0, m)   # per-axis cut-off from 10 eta
    assert np.linalg.norm(I - ref) / np.linalg.norm(ref) < 1e-5
    tri = np.array(box)
    tri[0, 1] = 1.0
    with pytest.raises(ValueError):
        oracle.fft_intensity(pos, f, tri, 32, 0.3, 10, m)
