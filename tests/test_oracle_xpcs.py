"""Pins of the oracle's g2 and XSVS contrast (arXiv 2204.13241 Sec. 2.3):
hand-computed series (tests/golden), closed forms of periodic and constant
signals, the Erlang 1/K law (Sec. 4.3) and the Brownian ideal gas
(Eqs. fq_exp, g2_from_fq, beta_alt_int in discrete form)."""
import math
import os

import numpy as np

import oracle
from paper_2204_13241_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_g2_hand_series():
    rows = _read("g2_hand.txt")
    series = {r[1]: [float(x) for x in r[2:]] for r in rows if r[0] == "I"}
    I = np.array([series["A"], series["B"]]).T  # [T][2]
    g, mean = oracle.g2(I, [0, 1, 2, 3])
    col = {"A": 0, "B": 1}
    for r in rows:
        if r[0] == "g2":
            assert abs(g[int(r[2]), col[r[1]]] - float(r[3])) < 1e-15
        if r[0] == "mean":
            assert abs(mean[col[r[1]]] - float(r[2])) < 1e-15


def test_g2_constant_and_periodic_closed_forms():
    T = 240
    t = np.arange(T)
    const = np.full((T, 3), 2.5)
    g, _ = oracle.g2(const, [0, 1, 17, 239])
    assert np.allclose(g, 1.0, rtol=1e-14)
    # I(t) = 1 + cos(2 pi t / P): over whole periods the mean is 1 and
    # <I(t) I(t+tau)> = 1 + cos(2 pi tau / P) / 2
    Pd = 12
    I = (1 + np.cos(2 * math.pi * t / Pd))[:, None]
    taus = [tau for tau in range(0, T) if (T - tau) % Pd == 0][:10]
    g, mean = oracle.g2(I, taus)
    assert abs(mean[0] - 1.0) < 1e-13
    ref = 1 + np.cos(2 * math.pi * np.array(taus) / Pd) / 2
    assert np.allclose(g[:, 0], ref, atol=1e-12)


def test_xsvs_hand_series():
    rows = _read("xsvs_hand.txt")
    frames = np.array([[float(x) for x in r[2:]] for r in rows if r[0] == "frame"])
    rings = np.array([int(x) for x in next(r for r in rows if r[0] == "rings")[1:]])
    beta, counts = oracle.xsvs_contrast(frames, [1, 2, 3], rings, 2)
    for r in rows:
        if r[0] == "beta":
            K, ring, val = int(r[1]), int(r[2]), float(r[3])
            assert abs(beta[K - 1, ring - 1] - val) < 1e-14
        if r[0] == "count":
            assert counts[int(r[1]) - 1] == int(r[2])


def test_xsvs_drops_partial_window_and_constant_gives_zero():
    T, P = 7, 5
    I = np.ones((T, P)) * 3.0
    rings = np.array([1, 1, 2, 2, 2])
    beta, _ = oracle.xsvs_contrast(I, [1, 2, 3, 7], rings, 2)
    assert np.allclose(beta, 0.0, atol=1e-15)
    # a spike in the dropped tail (t = 6 for K = 2 and 3) must not matter
    I2 = I.copy()
    I2[6, 0] = 1e6
    b2, _ = oracle.xsvs_contrast(I2, [2, 3], rings, 2)
    assert np.allclose(b2, 0.0, atol=1e-15)


def test_ring_assignment_against_bruteforce():
    grid = wl.centered_plane(32)
    L = 23.0
    m = grid.miller()
    r = oracle.ring_index(np.eye(3) * L, m, 1.0, 30)
    mag = np.sqrt((m.astype(np.float64) ** 2).sum(axis=1))
    for k in range(m.shape[0]):
        want = 0
        for ring in range(1, 31):
            if ring - 0.5 <= mag[k] < ring + 0.5:
                want = ring
        assert r[k] == want
    # narrow rings keep only pixels within w/2 of the centre
    r2 = oracle.ring_index(np.eye(3) * L, m, 0.4, 30)
    keep = r2 > 0
    assert np.all(np.abs(mag[keep] - r2[keep]) < 0.2 + 1e-12)
    assert np.all((np.abs(mag[~keep] - np.round(mag[~keep])) >= 0.2 - 1e-12) | (mag[~keep] < 0.8) | (mag[~keep] >= 30.5))


def test_erlang_contrast_of_independent_speckles():
    # sums of K independent fully developed speckle patterns: beta = beta0 / K,
    # beta0 = 1 - sum f^4 / (sum f^2)^2  (Sec. 4.3, Eq. Erlang)
    rng = np.random.default_rng(11)
    N, L, T = 300, 24.0, 24
    pos = (rng.random((T, N, 3)) * L).astype(np.float32)
    f = np.ones(N)
    grid = wl.centered_plane(24)
    m = grid.miller()
    I = oracle.intensity(pos, f, np.eye(3) * L, m)
    rings = oracle.ring_index(np.eye(3) * L, m, 1.0, 16)
    # pool rings 4..16 for statistics: one pseudo-ring
    pooled = np.where(rings >= 4, 1, 0)
    beta0 = 1 - (f ** 4).sum() / (f ** 2).sum() ** 2
    Ks = [1, 2, 4, 8]
    beta, counts = oracle.xsvs_contrast(I, Ks, pooled, 1)
    n_eff = counts[0]
    for k, K in enumerate(Ks):
        W = T // K
        tol = 6 * math.sqrt(2.0 / (n_eff * W)) / K + 0.02 / K
        assert abs(beta[k, 0] - beta0 / K) < tol, (K, beta[k, 0])


def test_brownian_ideal_gas_g2_and_contrast_closed_forms():
    # independent atoms diffusing along x only, sigma per frame:
    # F(q,tau) = exp(-q_x^2 sigma^2 tau / 2) = exp(-D q_x^2 tau), D = sigma^2 / 2,
    # the same for every pixel of a fixed n_x, so whole (n_y, n_z) planes pool.
    # g2 - 1 = beta0 |F|^2 (Siegert, Eq. g2_from_fq) and, for sums of K frames,
    # beta_K = beta0 / K^2 * sum_{i,j<K} |F(|i-j|)|^2 (discrete Eq. beta_alt_int).
    # Decay times are far below T so that the time averages converge.
    rng = np.random.default_rng(77)
    N, L, T, sigma = 256, 16.0, 800, 0.4
    base = rng.random((N, 3)) * L
    steps = np.zeros((T, N, 3))
    steps[1:, :, 0] = rng.standard_normal((T - 1, N)) * sigma
    pos = (base[None] + np.cumsum(steps, axis=0)).astype(np.float32)
    f = np.ones(N)
    planes = {nx: wl.QGrid(nx, 1, -7, 15, -7, 15).miller() for nx in (2, 3)}
    ms = np.concatenate(list(planes.values()))
    I = oracle.intensity(pos, f, np.eye(3) * L, ms)            # [T][450]
    D = sigma ** 2 / 2
    beta0 = 1 - 1.0 / N
    taus = [1, 2, 4, 8]
    g, _ = oracle.g2(I, taus)
    off = 0
    for nx, pl in planes.items():
        cols = np.arange(off, off + pl.shape[0])
        off += pl.shape[0]
        q2 = (2 * math.pi * nx / L) ** 2
        for it, tau in enumerate(taus):
            est = g[it, cols].mean() - 1
            ref = beta0 * math.exp(-2 * D * q2 * tau)
            se = g[it, cols].std() / math.sqrt(len(cols))
            assert abs(est - ref) < 5 * se + 0.01, (nx, tau, est, ref)
    # contrast of K-frame sums on the n_x = 2 plane pooled as one ring; the
    # finite-ring estimator bias is about 3 / 225, inside the 5 % band
    q2 = (2 * math.pi * 2 / L) ** 2
    pooled = np.zeros(ms.shape[0], dtype=np.int32)
    pooled[: planes[2].shape[0]] = 1
    Ks = [1, 3, 6]
    beta, _ = oracle.xsvs_contrast(I, Ks, pooled, 1)
    for k, K in enumerate(Ks):
        ref = beta0 / K ** 2 * sum(math.exp(-2 * D * q2 * abs(i - j)) for i in range(K) for j in range(K))
        assert abs(beta[k, 0] - ref) < 0.05 * ref, (K, beta[k, 0], ref)
