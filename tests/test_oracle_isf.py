"""Pins of the oracle's intermediate scattering function and of the contrast
it predicts (arXiv 2204.13241 Sec. 2.3, Eqs. fq_def_pos, Fq_pq, norm_Fq,
g2_from_fq, fq_exp and beta_alt_int):
  * the hand-worked series in tests/golden/isf_hand.txt;
  * the atom-pair double sum of Eq. fq_def_pos, by brute force on tiny
    trajectories (fixes the conjugation and the sum f^2 normalisation);
  * a static configuration, where F_hat = 1 and the contrast ratio is 1;
  * the pair-count form of the K-frame sum against the explicit double sum;
  * the closed form of an AR(1) Gaussian field, F_hat = rho^tau;
  * the Brownian ideal gas: F_hat = exp(-D q^2 tau), the Siegert relation
    g2 - 1 = beta0 |F_hat|^2, and the XSVS contrast equal to beta0 times
    the contrast predicted from F_hat."""
import math
import os

import numpy as np

import oracle
from paper_2204_13241_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [l.split() for l in fh if l.strip() and not l.startswith("#")]


def test_isf_hand_series():
    rows = _rows("isf_hand.txt")
    sumf2 = float(next(r for r in rows if r[0] == "sumf2")[1])
    S = {}
    for r in rows:
        if r[0] == "S":
            v = [float(x) for x in r[2:]]
            S[r[1]] = [complex(v[2 * i], v[2 * i + 1]) for i in range(len(v) // 2)]
    amp = np.array([S["A"], S["B"]]).T  # [T][2]
    col = {"A": 0, "B": 1}
    F, Fh = oracle.isf(amp, [0, 1, 2, 3], sumf2)
    for r in rows:
        if r[0] == "F":
            assert abs(F[int(r[2]), col[r[1]]] - complex(float(r[3]), float(r[4]))) < 1e-15
        if r[0] == "Fhat":
            assert abs(Fh[int(r[2]), col[r[1]]] - complex(float(r[3]), float(r[4]))) < 1e-15
    b, counts = oracle.contrast_from_isf(Fh, [1, 2, 3, 4], np.array([1, 2]), 2)
    assert list(counts) == [1, 1]
    for r in rows:
        if r[0] == "beta":
            assert abs(b[int(r[2]) - 1, col[r[1]]] - float(r[3])) < 1e-15


def test_isf_equals_atom_pair_double_sum():
    rng = np.random.default_rng(11)
    N, T, L = 5, 7, 6.0
    pos = (rng.random((T, N, 3)) * L).astype(np.float32)
    f = np.array([1.0, 0.6, 1.3, 0.6, 1.0])
    box = np.eye(3) * L
    m = np.array([[1, 0, 0], [2, -1, 3], [0, 0, 0], [-3, 2, 1]], dtype=np.int32)
    q = oracle.qvectors(box, m)
    taus = [0, 1, 3, 6]
    F, _ = oracle.isf(oracle.amplitude(pos, f, box, m), taus, float((f * f).sum()))
    r = pos.astype(np.float64)
    for k, tau in enumerate(taus):
        for ip in range(m.shape[0]):
            acc = 0j
            for t in range(T - tau):
                for i in range(N):
                    for j in range(N):
                        acc += f[i] * f[j] * np.exp(-1j * (q[ip] @ (r[t, i] - r[t + tau, j])))
            ref = acc / (T - tau) / (f * f).sum()
            assert abs(F[k, ip] - ref) < 1e-12 * max(1.0, abs(ref)), (tau, ip)


def test_static_configuration_has_unit_isf_and_contrast():
    rng = np.random.default_rng(12)
    pos = np.repeat((rng.random((1, 40, 3)) * 9.0).astype(np.float32), 20, axis=0)
    f = np.ones(40)
    m = wl.centered_plane(8).miller()
    S = oracle.amplitude(pos, f, np.eye(3) * 9.0, m)
    _, Fh = oracle.isf(S, list(range(20)), 40.0)
    nz = np.abs(S[0]) > 1e-9
    assert np.allclose(Fh[:, nz], 1.0, atol=1e-12)
    rings = oracle.ring_index(np.eye(3) * 9.0, m, 1.0, 5)
    keep = nz & (rings > 0)
    b, _ = oracle.contrast_from_isf(Fh[:, keep], [1, 2, 7, 20], rings[keep], 5)
    assert np.allclose(b[~np.isnan(b)], 1.0, atol=1e-12)


def test_pair_count_form_equals_double_sum():
    rng = np.random.default_rng(13)
    Fh = rng.standard_normal((9, 4)) + 1j * rng.standard_normal((9, 4))
    Fh[0] = 1.0
    rings = np.array([1, 1, 2, 3])
    b, _ = oracle.contrast_from_isf(Fh, [1, 2, 5, 9], rings, 3)
    a = np.abs(Fh) ** 2
    for ik, K in enumerate([1, 2, 5, 9]):
        per = np.array([sum(a[abs(i - j), p] for i in range(K) for j in range(K)) / K ** 2 for p in range(4)])
        ref = [per[:2].mean(), per[2], per[3]]
        assert np.allclose(b[ik], ref, rtol=1e-14)


def test_ar1_field_closed_forms():
    # a(t) = rho a(t-1) + sqrt(1 - rho^2) xi(t): F_hat(tau) = rho^tau, and the
    # K-frame contrast sum_{i,j<K} rho^(2|i-j|) / K^2 has the closed form
    # [K (1 + x) / (1 - x) - 2 x (1 - x^K) / (1 - x)^2] / K^2, x = rho^2
    rho, T, P = 0.8, 4000, 400
    rng = np.random.default_rng(14)
    a = np.empty((T, P), dtype=np.complex128)
    a[0] = (rng.standard_normal(P) + 1j * rng.standard_normal(P)) / math.sqrt(2)
    s = math.sqrt(1 - rho * rho)
    for t in range(1, T):
        a[t] = rho * a[t - 1] + s * (rng.standard_normal(P) + 1j * rng.standard_normal(P)) / math.sqrt(2)
    _, Fh = oracle.isf(a, [0, 1, 2, 3], 1.0)
    for k in range(4):
        est = Fh[k].mean()
        assert abs(est - rho ** k) < 5 * Fh[k].std() / math.sqrt(P) + 0.01, (k, est)
    Fexact = np.array([rho ** d for d in range(50)], dtype=np.complex128)[:, None]
    b, _ = oracle.contrast_from_isf(Fexact, [1, 3, 10, 50], np.array([1]), 1)
    x = rho * rho
    for ik, K in enumerate([1, 3, 10, 50]):
        ref = (K * (1 + x) / (1 - x) - 2 * x * (1 - x ** K) / (1 - x) ** 2) / K ** 2
        assert abs(b[ik, 0] - ref) < 1e-13


def test_brownian_gas_isf_siegert_and_contrast():
    # independent Brownian atoms, x steps only: F_hat(n,tau) = exp(-D q_x^2 tau)
    # on whole (n_y, n_z) planes of fixed n_x (Eq. fq_exp); the Siegert
    # relation gives g2 - 1 = beta0 |F_hat|^2 with beta0 = 1 - sum f^4/(sum f^2)^2
    N, T, L, sig = 400, 3000, 20.0, 0.35
    rng = np.random.default_rng(15)
    base = rng.random((N, 3)) * L
    steps = np.zeros((T, N, 3))
    steps[1:, :, 0] = rng.standard_normal((T - 1, N)) * sig
    pos = (base[None] + np.cumsum(steps, axis=0)).astype(np.float32)
    f = np.ones(N)
    D = sig * sig / 2
    grid = wl.QGrid(1, 4, -3, 7, -3, 7)
    m = grid.miller()
    S = oracle.amplitude(pos, f, np.eye(3) * L, m)
    taus = [1, 2, 4]
    _, Fh = oracle.isf(S, taus, float(N))
    I = S.real ** 2 + S.imag ** 2
    g, _ = oracle.g2(I, taus)
    beta0 = 1 - 1.0 / N
    for nx in range(1, 5):
        sel = m[:, 0] == nx
        q2 = (2 * math.pi * nx / L) ** 2
        for k, tau in enumerate(taus):
            want = math.exp(-D * q2 * tau)
            est = Fh[k, sel].real.mean()
            se = Fh[k, sel].real.std() / math.sqrt(sel.sum())
            assert abs(est - want) < 5 * se + 0.02, (nx, tau, est, want)
            sieg = (g[k, sel] - 1).mean() / beta0
            assert abs(sieg - np.abs(Fh[k, sel]).mean() ** 2) < 0.05 + 5 * (g[k, sel] - 1).std() / math.sqrt(sel.sum())
    # XSVS contrast of K-frame exposures against the contrast predicted from
    # F_hat, per n_x plane.  Both are taken relative to K = 1, which removes
    # the finite-ring bias of the XSVS estimate (49 pixels per plane) and beta0.
    Kmax = 6
    _, Fd = oracle.isf(S, list(range(Kmax)), float(N))
    planes = m[:, 0]
    bI, _ = oracle.xsvs_contrast(I, [1, 2, 3, 6], planes, 4)
    bF, _ = oracle.contrast_from_isf(Fd, [1, 2, 3, 6], planes, 4)
    assert np.allclose(bF[0], 1.0)
    assert np.allclose(bI / bI[0], bF, rtol=0.02), (bI / bI[0], bF)
    assert bF[3, 3] < 0.75   # the slowest plane decorrelates within 6 frames
