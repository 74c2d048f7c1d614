"""FP64 CPU oracle of the direct-method XPCS/XSVS path -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the bench's CPU-baseline leg may import
this package.  It shares no code with the CUDA library: the intensity is the
plain C direct sum in ``direct.c`` (built by :func:`build`), the correlation
stages are written out below in numpy float64.

What each function follows (arXiv 2204.13241):
  amplitude / intensity   Sec. 2.2 Eqs. pe_ri, Iq_pq; Sec. 3.1 Eq.
                          sq_cut_simple and Algorithm 1 (direct method).
  form_factor, amplitude_species, intensity_species
                          Sec. 2.1: per-atom form factors f_i(q), each a sum
                          of Gaussians in |q| for its species.
  fft_intensity           Sec. 3.2 Algorithm 2 (Gaussian-smeared density on a
                          grid, FFT, division by the transform of one
                          Gaussian), the paper's FFT method as a cross-check.
  ewald_points            the spherical detector slice |k_f| = |k_i| (Fig. 5,
                          Sec. 4.5), as reciprocal-lattice points.
  g2                      Sec. 2.3 Eq. g2_def (XPCS autocorrelation).
  ring_index, xsvs_contrast
                          Sec. 2.3 Eqs. inte_Iq and bq_Iq (finite-exposure
                          intensity as a sum of K frames, optical contrast
                          over a |q| ring), averaged over exposures (Sec. 4.3).
  isf, contrast_from_isf  Sec. 2.3 Eqs. Fq_pq and norm_Fq (intermediate
                          scattering function from the amplitudes) and Eq.
                          beta_alt_int (contrast predicted through the
                          Siegert relation, in its K-frame form).
  grad_analytic           derivative of I = |S|^2 with respect to the atomic
                          positions (the adjoint of Eq. pe_ri).
  grad_fd                 central finite differences of a caller loss, with an
                          exact incremental update of S per displaced atom.

Readings taken where the paper leaves a choice: S uses exp(+i q.r) (the
paper's p^e is its conjugate; I is the same); g2's numerator averages the T - tau available products and its
denominator is the square of the mean over all T frames; a ring r holds the
pixels with r - w/2 <= |q|/Delta < r + w/2, Delta = 2 pi / det(h)^(1/3);
windows are the floor(T/K) non-overlapping blocks of K frames and beta is the
population contrast averaged over windows.

Every function here is pinned in tests/test_oracle_*.py against closed forms,
invariants, brute force or hand-computed values; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile direct.c into _build/liboracle.so with gcc (FP64, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "direct.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_amplitude.argtypes = [P, I64, I64, P, P, P, I64, P, ctypes.c_int]
        lib.oracle_amplitude.restype = ctypes.c_int
        lib.oracle_qvectors.argtypes = [P, P, I64, P]
        lib.oracle_qvectors.restype = ctypes.c_int
        lib.oracle_inverse3.argtypes = [P, P]
        lib.oracle_inverse3.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ----------------------------------------------------------------------------
# intensity (direct method)
# ----------------------------------------------------------------------------

def qvectors(box: np.ndarray, miller: np.ndarray) -> np.ndarray:
    """q = 2 pi h^-T n for each Miller index, float64 [P][3]."""
    h = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    m = np.ascontiguousarray(miller, dtype=np.int32).reshape(-1, 3)
    out = np.empty((m.shape[0], 3), dtype=np.float64)
    if not _load().oracle_qvectors(_ptr(h), _ptr(m), m.shape[0], _ptr(out)):
        raise ValueError("singular cell matrix")
    return out


def amplitude(pos: np.ndarray, f: np.ndarray, box: np.ndarray, miller: np.ndarray,
              threads: int = 0) -> np.ndarray:
    """S(q,t) = sum_j f_j exp(+i q.r_j(t)), complex128 [T][P].

    `pos` float32 [T][N][3] (or [N][3] for one frame), `f` [N], `box` 3x3
    (columns = cell edge vectors), `miller` int [P][3]."""
    p = np.ascontiguousarray(pos, dtype=np.float32)
    if p.ndim == 2:
        p = p[None]
    T, N, _ = p.shape
    fd = np.ascontiguousarray(f, dtype=np.float64).reshape(N)
    h = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    m = np.ascontiguousarray(miller, dtype=np.int32).reshape(-1, 3)
    out = np.empty((T, m.shape[0], 2), dtype=np.float64)
    ok = _load().oracle_amplitude(_ptr(p), N, T, _ptr(fd), _ptr(h), _ptr(m), m.shape[0],
                                  _ptr(out), int(threads))
    if not ok:
        raise ValueError("singular cell matrix")
    return out[..., 0] + 1j * out[..., 1]


def intensity(pos, f, box, miller, threads: int = 0) -> np.ndarray:
    """I(q,t) = |S(q,t)|^2, float64 [T][P]."""
    s = amplitude(pos, f, box, miller, threads)
    return s.real ** 2 + s.imag ** 2


# ----------------------------------------------------------------------------
# q-dependent form factors of several atom species
# ----------------------------------------------------------------------------

def form_factor(coef: np.ndarray, qnorm: np.ndarray) -> np.ndarray:
    """f(q) as a sum of Gaussians (Sec. 2.1): with s = |q| / (4 pi),
    f = sum_{k<4} a_k exp(-b_k s^2) + c, coef = (a1, b1, a2, b2, a3, b3, a4, b4, c).
    Returns float64 shaped like qnorm."""
    c = np.asarray(coef, dtype=np.float64).reshape(9)
    s2 = (np.asarray(qnorm, dtype=np.float64) / (4.0 * math.pi)) ** 2
    out = np.full(s2.shape, c[8])
    for k in range(4):
        out = out + c[2 * k] * np.exp(-c[2 * k + 1] * s2)
    return out


def amplitude_species(pos, f, species, coef, box, miller, threads: int = 0) -> np.ndarray:
    """S(q,t) = sum_j f_j F_{s_j}(q) exp(+i q.r_j(t)) (Sec. 2.1 with per-atom
    form factors f_i(q)); f_j is a per-atom weight, F_s the Gaussian-sum form
    factor of species s (`coef` [n_species][9]).  The sum is grouped by
    species: each group is the plain direct sum of its atoms, scaled by its
    F_s(q).  complex128 [T][P]."""
    sp = np.asarray(species).reshape(-1)
    cf = np.asarray(coef, dtype=np.float64).reshape(-1, 9)
    fw = np.asarray(f, dtype=np.float64).reshape(-1)
    qn = np.sqrt((qvectors(box, miller) ** 2).sum(axis=1))
    total = None
    for s_id in range(cf.shape[0]):
        part = amplitude(pos, np.where(sp == s_id, fw, 0.0), box, miller, threads)
        part = part * form_factor(cf[s_id], qn)[None, :]
        total = part if total is None else total + part
    return total


def intensity_species(pos, f, species, coef, box, miller, threads: int = 0) -> np.ndarray:
    """|S|^2 of :func:`amplitude_species`, float64 [T][P]."""
    s = amplitude_species(pos, f, species, coef, box, miller, threads)
    return s.real ** 2 + s.imag ** 2


# ----------------------------------------------------------------------------
# the FFT-based method (Algorithm 2), a cross-check of the direct sum
# ----------------------------------------------------------------------------

def _nearest_points(x: float, k: int) -> np.ndarray:
    """Indices of the k grid points nearest to x (in grid units)."""
    return math.ceil(x - k / 2.0) + np.arange(k)


def fft_intensity(pos, f, box, n_grid: int, eta: float, k_cut: int, miller) -> np.ndarray:
    """I(q,t) by Algorithm 2 (Sec. 3.2) on an n_grid^3 grid of an
    orthorhombic cell, at the Miller indices `miller` (|n_a| <= n_grid / 2):
      rho(r) = sum_i f_i (2 pi eta^2)^(-3/2) exp(-|r - r_i|^2 / (2 eta^2)) on the
               k_cut^3 grid points nearest each atom (periodic images; k_cut <= 0
               takes the smallest integer above 10 eta per axis);
      p^eta(q) = FFT of rho (times the cell volume per grid point);
      f^eta(q) = the same transform of one Gaussian centred at the origin and
               truncated the same way;
      I = |p^eta / f^eta|^2 (Eq. Iq_pq_new with the per-atom f_i inside rho).
    numpy's FFT is the library step; float64 throughout; [T][P]."""
    h = np.asarray(box, dtype=np.float64).reshape(3, 3)
    if np.count_nonzero(h - np.diag(np.diag(h))):
        raise ValueError("Algorithm 2 here takes an orthorhombic cell")
    Ls = np.diag(h)
    hg = Ls / n_grid                                   # grid spacing per axis
    p3 = np.asarray(pos, dtype=np.float64)
    if p3.ndim == 2:
        p3 = p3[None]
    fw = np.asarray(f, dtype=np.float64).reshape(-1)
    norm = (2.0 * math.pi * eta * eta) ** -1.5
    dv = float(np.prod(hg))

    # k_cut <= 0: per axis the smallest integer above 10 eta in grid steps (the
    # paper's rule, which keeps +-5 eta around each atom)
    ks = [int(k_cut) if k_cut > 0 else int(math.floor(10.0 * eta / hg[a])) + 1 for a in range(3)]

    def gauss_1d(x0, a):
        idx = _nearest_points(x0 / hg[a], ks[a])
        w = np.exp(-((idx * hg[a] - x0) ** 2) / (2.0 * eta * eta))
        return idx % n_grid, w

    # f^eta: the truncated origin Gaussian is a product of 1D factors
    feta = np.ones((n_grid,) * 3, dtype=np.complex128)
    for a in range(3):
        idx, w = gauss_1d(0.0, a)
        line = np.zeros(n_grid)
        np.add.at(line, idx, w)
        shape = [1, 1, 1]
        shape[a] = n_grid
        feta = feta * np.fft.fft(line).reshape(shape)
    feta = feta * norm * dv
    m = np.asarray(miller, dtype=np.int64).reshape(-1, 3) % n_grid
    out = np.empty((p3.shape[0], m.shape[0]), dtype=np.float64)
    for t in range(p3.shape[0]):
        rho = np.zeros((n_grid,) * 3)
        for i in range(p3.shape[1]):
            ix, wx = gauss_1d(p3[t, i, 0], 0)
            iy, wy = gauss_1d(p3[t, i, 1], 1)
            iz, wz = gauss_1d(p3[t, i, 2], 2)
            blk = fw[i] * norm * wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
            rho[np.ix_(ix, iy, iz)] += blk
        P = np.fft.fftn(rho) * dv                     # exp(-i q.r), index order (x, y, z)
        v = P[m[:, 0], m[:, 1], m[:, 2]] / feta[m[:, 0], m[:, 1], m[:, 2]]
        out[t] = v.real ** 2 + v.imag ** 2
    return out


# ----------------------------------------------------------------------------
# detector pixels on the Ewald sphere
# ----------------------------------------------------------------------------

def ewald_points(box: np.ndarray, k_in, nx0: int, nx: int, ny0: int, ny: int
                 ) -> tuple[np.ndarray, np.ndarray]:
    """Reciprocal-lattice points on the Ewald sphere for a detector window of
    (n_x, n_y) (the spherical slice of Fig. 5: |k_f| = |k_i| with
    k_f = k_i + q).  For each (n_x, n_y), q(n_z) = 2 pi h^-T (n_x, n_y, n_z) is
    a line in n_z; it meets the sphere |q + k_i| = |k_i| at the real roots of
    |q + k_i|^2 = |k_i|^2.  The root nearer n_z = 0 is kept, and of the two
    integers around it the one whose q lies closer to the sphere (ties: the
    smaller |n_z|).  Returns (miller int32 [nx*ny][3], x fastest, and valid
    bool [nx*ny]; a line that misses the sphere is invalid)."""
    h = np.asarray(box, dtype=np.float64).reshape(3, 3)
    Ht = 2.0 * math.pi * np.linalg.inv(h).T          # q = Ht n
    k = np.asarray(k_in, dtype=np.float64).reshape(3)
    kk = float(k @ k)
    yy, xx = np.meshgrid(np.arange(ny0, ny0 + ny), np.arange(nx0, nx0 + nx), indexing="ij")
    xx, yy = xx.ravel(), yy.ravel()
    q0 = np.stack([xx, yy, np.zeros_like(xx)], axis=1).astype(np.float64) @ Ht.T
    d = Ht[:, 2]
    A = float(d @ d)
    B = 2.0 * (q0 @ d + float(d @ k))
    C = (q0 * q0).sum(axis=1) + 2.0 * (q0 @ k)
    disc = B * B - 4.0 * A * C
    valid = disc >= 0.0
    sq = np.sqrt(np.where(valid, disc, 0.0))
    r1 = (-B + sq) / (2.0 * A)
    r2 = (-B - sq) / (2.0 * A)
    root = np.where(np.abs(r1) <= np.abs(r2), r1, r2)

    def dist(nz):
        q = q0 + nz[:, None] * d[None, :]
        return np.abs(np.sqrt(((q + k) ** 2).sum(axis=1)) - math.sqrt(kk))

    lo, hi = np.floor(root), np.ceil(root)
    dl, dh = dist(lo), dist(hi)
    pick = np.where((dl < dh) | ((dl == dh) & (np.abs(lo) <= np.abs(hi))), lo, hi)
    nz = np.where(valid, pick, 0.0).astype(np.int64)
    m = np.stack([xx, yy, nz], axis=1).astype(np.int32)
    return m, valid


# ----------------------------------------------------------------------------
# XPCS autocorrelation
# ----------------------------------------------------------------------------

def g2(I: np.ndarray, taus: Sequence[int]) -> tuple[np.ndarray, np.ndarray]:
    """g2(q,tau) = <I(t) I(t+tau)>_t / <I(t)>_t^2 per pixel.

    I [T][P]; the numerator averages the T - tau products with t in
    [0, T - tau), the denominator squares the mean over all T frames.
    Returns (g2 float64 [n_tau][P], mean float64 [P])."""
    x = np.asarray(I, dtype=np.float64)
    T = x.shape[0]
    mean = x.sum(axis=0) / T
    out = np.empty((len(taus),) + x.shape[1:], dtype=np.float64)
    for k, tau in enumerate(taus):
        tau = int(tau)
        if tau < 0 or tau >= T:
            raise ValueError("delay out of range")
        num = (x[: T - tau] * x[tau:]).sum(axis=0) / (T - tau)
        with np.errstate(divide="ignore", invalid="ignore"):
            out[k] = num / (mean * mean)
    return out, mean


# ----------------------------------------------------------------------------
# XSVS contrast
# ----------------------------------------------------------------------------

def ring_index(box: np.ndarray, miller: np.ndarray, ring_width: float, n_rings: int) -> np.ndarray:
    """Ring of each pixel (1..n_rings) or 0 when the pixel is in no ring.

    Ring r collects r - w/2 <= |q|/Delta < r + w/2 with Delta = 2 pi /
    det(h)^(1/3) (= 2 pi / L for a cubic box)."""
    q = qvectors(box, miller)
    det = float(np.linalg.det(np.asarray(box, dtype=np.float64)))
    delta = 2.0 * math.pi / abs(det) ** (1.0 / 3.0)
    x = np.sqrt((q * q).sum(axis=1)) / delta
    r = np.floor(x + 0.5)
    ok = (r >= 1) & (r <= n_rings) & (x >= r - ring_width / 2.0) & (x < r + ring_width / 2.0)
    return np.where(ok, r, 0).astype(np.int32)


def xsvs_contrast(I: np.ndarray, Ks: Sequence[int], rings: np.ndarray, n_rings: int
                  ) -> tuple[np.ndarray, np.ndarray]:
    """beta_K(r), float64 [n_K][n_rings], and pixels per ring.

    For window length K the exposures are I_K(q,w) = sum_{t=wK}^{wK+K-1}
    I(q,t), w = 0..floor(T/K)-1; per window and ring
    beta = (<I_K^2>_ring - <I_K>_ring^2) / <I_K>_ring^2, then beta_K(r) is the
    mean of beta over windows.  A ring with no pixel gives NaN."""
    x = np.asarray(I, dtype=np.float64)
    T = x.shape[0]
    rings = np.asarray(rings).reshape(-1)
    counts = np.array([(rings == r).sum() for r in range(1, n_rings + 1)], dtype=np.int64)
    out = np.full((len(Ks), n_rings), np.nan, dtype=np.float64)
    for ik, K in enumerate(Ks):
        K = int(K)
        if K < 1 or K > T:
            raise ValueError("window length out of range")
        W = T // K
        sums = np.stack([x[w * K:(w + 1) * K].sum(axis=0) for w in range(W)])  # [W][P]
        for r in range(1, n_rings + 1):
            sel = rings == r
            n = int(sel.sum())
            if n == 0:
                continue
            v = sums[:, sel]
            m1 = v.sum(axis=1) / n
            m2 = (v * v).sum(axis=1) / n
            with np.errstate(divide="ignore", invalid="ignore"):
                beta_w = (m2 - m1 * m1) / (m1 * m1)
            out[ik, r - 1] = beta_w.sum() / W
    return out, counts


# ----------------------------------------------------------------------------
# intermediate scattering function and the contrast it predicts
# ----------------------------------------------------------------------------

def isf(S: np.ndarray, taus: Sequence[int], sum_f2: float) -> tuple[np.ndarray, np.ndarray]:
    """F(q,tau) and F_hat(q,tau), complex128 [n_tau][P] each.

    F = <p(t) p*(t+tau)>_t / sum_j f_j^2 (Sec. 2.3 Eq. Fq_pq) with p the
    conjugate of S, so the product is conj(S(t)) S(t+tau), averaged over the
    T - tau available t; F_hat = F / F(q,0) (Eq. norm_Fq) with F(q,0) the mean
    of |S|^2 over all T frames divided by sum_j f_j^2."""
    x = np.asarray(S, dtype=np.complex128)
    T = x.shape[0]
    F0 = (x.real ** 2 + x.imag ** 2).sum(axis=0) / T / float(sum_f2)
    F = np.empty((len(taus),) + x.shape[1:], dtype=np.complex128)
    for k, tau in enumerate(taus):
        tau = int(tau)
        if tau < 0 or tau >= T:
            raise ValueError("delay out of range")
        F[k] = (np.conj(x[: T - tau]) * x[tau:]).sum(axis=0) / (T - tau) / float(sum_f2)
    with np.errstate(divide="ignore", invalid="ignore"):
        Fhat = F / F0
    return F, Fhat


def contrast_from_isf(Fhat_dense: np.ndarray, Ks: Sequence[int], rings: np.ndarray, n_rings: int
                      ) -> tuple[np.ndarray, np.ndarray]:
    """beta_K / beta_0 per ring predicted from |F_hat|^2 through the Siegert
    relation (Sec. 2.3 Eq. beta_alt_int), float64 [n_K][n_rings], and pixels
    per ring.

    Fhat_dense [Kmax][P] holds the delays 0 .. Kmax-1.  For an exposure that
    sums K frames the integral over the exposure becomes the double sum
    (1/K^2) sum_{i,j<K} |F_hat(|i-j|)|^2, with |F_hat(0)|^2 = 1 by definition;
    it is evaluated per pixel and averaged over the ring's pixels."""
    a = np.abs(np.asarray(Fhat_dense, dtype=np.complex128)) ** 2
    rings = np.asarray(rings).reshape(-1)
    counts = np.array([(rings == r).sum() for r in range(1, n_rings + 1)], dtype=np.int64)
    out = np.full((len(Ks), n_rings), np.nan, dtype=np.float64)
    for ik, K in enumerate(Ks):
        K = int(K)
        if K < 1 or K > a.shape[0]:
            raise ValueError("window length out of range")
        # (i, j) pairs with |i - j| = d: K for d = 0, 2 (K - d) for d >= 1
        per_pixel = np.full(a.shape[1:], float(K), dtype=np.float64)
        for d in range(1, K):
            per_pixel += 2.0 * (K - d) * a[d]
        per_pixel /= K * K
        for r in range(1, n_rings + 1):
            sel = rings == r
            if sel.any():
                out[ik, r - 1] = per_pixel[sel].mean()
    return out, counts


# ----------------------------------------------------------------------------
# gradients with respect to positions
# ----------------------------------------------------------------------------

def grad_analytic(pos: np.ndarray, f: np.ndarray, box: np.ndarray, miller: np.ndarray,
                  dL_dI: np.ndarray, atoms: Optional[np.ndarray] = None,
                  amp: Optional[np.ndarray] = None) -> np.ndarray:
    """dL/dr_j = sum_q dL/dI_q * 2 Re[conj(S_q) * i q f_j exp(i q.r_j)].

    One frame: pos [N][3].  `atoms` selects the rows returned (all by
    default); `amp` may pass S for the full atom set (else it is computed)."""
    p = np.asarray(pos, dtype=np.float32).reshape(-1, 3)
    q = qvectors(box, miller)
    if amp is None:
        amp = amplitude(p, f, box, miller)[0]
    H = np.asarray(dL_dI, dtype=np.float64).reshape(-1) * np.conj(amp)
    sel = np.arange(p.shape[0]) if atoms is None else np.asarray(atoms)
    fd = np.asarray(f, dtype=np.float64)
    out = np.empty((sel.size, 3), dtype=np.float64)
    for k0 in range(0, sel.size, 64):
        idx = sel[k0:k0 + 64]
        th = p[idx].astype(np.float64) @ q.T                    # [n][P]
        e = np.cos(th) + 1j * np.sin(th)
        val = 2.0 * fd[idx, None] * np.real(1j * H[None, :] * e)  # [n][P]
        out[k0:k0 + idx.size] = val @ q
    return out


def grad_fd(pos: np.ndarray, f: np.ndarray, box: np.ndarray, miller: np.ndarray,
            loss_of_I, atoms: Sequence[int], h: float = 1e-4,
            amp: Optional[np.ndarray] = None) -> np.ndarray:
    """Central differences (L(r + h e_a) - L(r - h e_a)) / 2h of loss_of_I(I).

    The displaced amplitude is S + f_j (exp(i q.r'_j) - exp(i q.r_j)),
    exact in FP64 and O(P) per displacement."""
    p = np.asarray(pos, dtype=np.float32).reshape(-1, 3)
    q = qvectors(box, miller)
    S = amplitude(p, f, box, miller)[0] if amp is None else np.asarray(amp)
    fd = np.asarray(f, dtype=np.float64)
    out = np.empty((len(atoms), 3), dtype=np.float64)
    for k, j in enumerate(atoms):
        r0 = p[j].astype(np.float64)
        e0 = np.exp(1j * (q @ r0))
        for a in range(3):
            vals = []
            for sgn in (+1.0, -1.0):
                r1 = r0.copy()
                r1[a] += sgn * h
                S1 = S + fd[j] * (np.exp(1j * (q @ r1)) - e0)
                vals.append(loss_of_I(S1.real ** 2 + S1.imag ** 2))
            out[k, a] = (vals[0] - vals[1]) / (2.0 * h)
    return out
