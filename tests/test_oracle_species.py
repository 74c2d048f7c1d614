"""Pins of the oracle's q-dependent, per-species form factors (arXiv
2204.13241 Sec. 2.1, Eq. Iq_rij with f_i(q)):
  * the Gaussian-sum form factor against hand values and its q = 0 limit;
  * the species-grouped amplitude against a per-atom brute force that
    evaluates f_i(q) exp(+i q.r_i) atom by atom;
  * one species with a constant form factor reduces to the plain amplitude;
  * a species with zero form factor drops out (tracer labelling, Sec. 4.5)."""
import math

import numpy as np

import oracle
from paper_2204_13241_gb300 import workloads as wl


def test_form_factor_hand_values():
    # f(s) = 2 exp(-3 s^2) + 0.5 exp(-0.25 s^2) + 0.75, s = |q| / (4 pi)
    coef = [2.0, 3.0, 0.5, 0.25, 0.0, 1.0, 0.0, 7.0, 0.75]
    q = np.array([0.0, 4 * math.pi, 2 * math.pi])
    got = oracle.form_factor(coef, q)
    assert abs(got[0] - 3.25) < 1e-15                                          # sum a + c
    assert abs(got[1] - (2 * math.exp(-3) + 0.5 * math.exp(-0.25) + 0.75)) < 1e-15   # s = 1
    assert abs(got[2] - (2 * math.exp(-0.75) + 0.5 * math.exp(-0.0625) + 0.75)) < 1e-15  # s = 1/2


def test_species_amplitude_equals_per_atom_brute_force():
    rng = np.random.default_rng(21)
    N, T, L = 23, 3, 7.5
    pos = (rng.random((T, N, 3)) * L).astype(np.float32)
    f = rng.random(N) + 0.5
    species = rng.integers(0, 3, N).astype(np.int32)
    coef = np.array([[1.0, 2.0, 0.3, 10.0, 0, 0, 0, 0, 0.1],
                     [4.0, 0.5, 1.0, 1.5, 2.0, 30.0, 0.5, 0.1, 1.2],
                     [0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0, 2.0]])
    box = np.eye(3) * L
    m = np.array([[0, 0, 0], [1, 2, 3], [-4, 0, 1], [7, -5, 2]], dtype=np.int32)
    S = oracle.amplitude_species(pos, f, species, coef, box, m)
    q = 2 * math.pi * m.astype(np.float64) / L
    qn = np.sqrt((q * q).sum(axis=1))
    for t in range(T):
        for ip in range(m.shape[0]):
            acc = 0j
            for j in range(N):
                c = coef[species[j]]
                s2 = (qn[ip] / (4 * math.pi)) ** 2
                ff = c[8] + sum(c[2 * k] * math.exp(-c[2 * k + 1] * s2) for k in range(4))
                acc += f[j] * ff * np.exp(1j * (q[ip] @ pos[t, j].astype(np.float64)))
            assert abs(S[t, ip] - acc) < 1e-12 * max(1.0, abs(acc))


def test_single_constant_species_is_plain_amplitude_and_zero_species_drops_out():
    traj, grid = wl.config0(keep=[0, 5])
    m = grid.miller()
    coef = np.array([[0, 0, 0, 0, 0, 0, 0, 0, 1.0]])
    S1 = oracle.amplitude_species(traj.pos, traj.f, np.zeros(traj.n_atoms, np.int32), coef, traj.box, m)
    S0 = oracle.amplitude(traj.pos, traj.f, traj.box, m)
    assert np.array_equal(S1, S0)
    # tracer labelling: 45 atoms of species 1 scatter, the rest (species 0) do not
    sp = np.zeros(traj.n_atoms, np.int32)
    sp[::89] = 1
    coef2 = np.array([[0, 0, 0, 0, 0, 0, 0, 0, 0.0], [0, 0, 0, 0, 0, 0, 0, 0, 1.0]])
    S2 = oracle.amplitude_species(traj.pos, traj.f, sp, coef2, traj.box, m)
    S3 = oracle.amplitude(traj.pos[:, sp == 1], traj.f[sp == 1], traj.box, m)
    assert np.allclose(S2, S3, rtol=0, atol=1e-12)
    assert (sp == 1).sum() == 45
