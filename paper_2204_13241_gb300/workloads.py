"""Seeded synthetic inputs for the direct-method XPCS/XSVS path.

This module only draws inputs: atomic positions of MD-like trajectories,
per-atom form factors, detector q-grids and the delay / window lists the
correlation stages are evaluated on.  It holds none of the method's
arithmetic (no phases, no sums over atoms, no intensities), so that the
CUDA path and the CPU oracle can both consume exactly the same arrays.

The paper's own inputs are MD trajectories of Lennard-Jones argon and
TIP4P/2005 water (Sec. 4.1, Sec. 4.6); they are not available, so the
workloads below stand in for them with the same kind of structure: a
periodic cubic box, positions in Angstrom, one snapshot per frame, and
reciprocal-lattice detector grids q = 2*pi*n/L (Sec. 3.1).

Conventions shared by every consumer:
  * positions are float32, shape [T][N][3], unwrapped (atoms may leave the
    box; the method is periodic so the image does not matter, Sec. 3.1);
  * form factors are float32 [N], constant in q;
  * the cell matrix `box` is float64 [3][3] whose COLUMNS are the cell edge
    vectors, so fractional coordinates are s = box^-1 r;
  * a detector grid is the Miller-index box
    n_x in [nx0, nx0+nx), n_y in [ny0, ny0+ny), n_z in [nz0, nz0+nz).

Random streams: NumPy PCG64 seeded with 2204132410 + config id, drawn in a
fixed order: lattice or uniform positions, thermal displacements,
vacancies, form factors, then the per-frame Brownian steps.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterable, Optional, Sequence

import numpy as np

SEED_BASE = 2204132410


@dataclasses.dataclass
class QGrid:
    """Miller-index ranges of a detector plane (nz == 1) or volume."""

    nx0: int
    nx: int
    ny0: int
    ny: int
    nz0: int = 0
    nz: int = 1

    @property
    def n_pixels(self) -> int:
        return self.nx * self.ny * self.nz

    def as_tuple(self):
        return (self.nx0, self.nx, self.ny0, self.ny, self.nz0, self.nz)

    def miller(self) -> np.ndarray:
        """Integer Miller indices [P][3] in output order (x fastest, then y, then z)."""
        z, y, x = np.meshgrid(
            np.arange(self.nz0, self.nz0 + self.nz),
            np.arange(self.ny0, self.ny0 + self.ny),
            np.arange(self.nx0, self.nx0 + self.nx),
            indexing="ij",
        )
        return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int32)


def centered_plane(side: int, nz: int = 0) -> QGrid:
    """Plane n_x, n_y in [-side/2, side/2 - 1] at fixed n_z."""
    return QGrid(-(side // 2), side, -(side // 2), side, nz, 1)


def centered_volume(side: int) -> QGrid:
    return QGrid(-(side // 2), side, -(side // 2), side, -(side // 2), side)


@dataclasses.dataclass
class Trajectory:
    pos: np.ndarray          # float32 [T_kept][N][3]
    f: np.ndarray            # float32 [N]
    box: np.ndarray          # float64 [3][3], columns = cell edge vectors
    frames: np.ndarray       # int64 frame indices held in pos
    n_frames_total: int      # frames in the full trajectory
    sigma_step: float = 0.0  # Brownian step per Cartesian component, Angstrom

    @property
    def n_atoms(self) -> int:
        return int(self.f.shape[0])

    @property
    def L(self) -> float:
        return float(self.box[0, 0])


def cubic_box(L: float) -> np.ndarray:
    return np.eye(3, dtype=np.float64) * float(L)


def fcc_sites(cells: int, a: float) -> np.ndarray:
    """Face-centred cubic sites of a cells^3 supercell, float64 [4*cells^3][3]."""
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    g = np.arange(cells, dtype=np.float64)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    corners = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (corners[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return sites * float(a)


def brownian_frames(rng: np.random.Generator, base: np.ndarray, n_frames: int, sigma: float,
                    keep: Optional[Iterable[int]] = None) -> tuple[np.ndarray, np.ndarray]:
    """Frame t = base + sum of t Gaussian steps (sigma per component).

    Steps are drawn frame after frame from `rng` (one [N][3] draw per frame
    1..T-1) so that any subset of frames is reproducible.  Accumulation is in
    float64; each kept frame is then rounded to float32.
    """
    n = base.shape[0]
    keep_idx = np.arange(n_frames) if keep is None else np.array(sorted(set(int(k) for k in keep)))
    if keep_idx.size and (keep_idx[0] < 0 or keep_idx[-1] >= n_frames):
        raise ValueError("frame index out of range")
    out = np.empty((keep_idx.size, n, 3), dtype=np.float32)
    cur = base.astype(np.float64, copy=True)
    slot = 0
    last = int(keep_idx[-1]) if keep_idx.size else -1
    for t in range(0, last + 1):
        if t > 0:
            cur += rng.standard_normal((n, 3)) * sigma
        if slot < keep_idx.size and keep_idx[slot] == t:
            out[slot] = cur
            slot += 1
    return out, keep_idx


def brownian_gas(seed: int, n_atoms: int, L: float, n_frames: int, sigma: float,
                 f_values: Sequence[float] = (1.0,), keep=None) -> Trajectory:
    """Ideal gas: uniform positions in [0, L)^3, then Brownian frames."""
    rng = np.random.default_rng(seed)
    base = rng.random((n_atoms, 3)) * L
    if len(f_values) == 1:
        f = np.full(n_atoms, f_values[0], dtype=np.float32)
    else:
        f = np.asarray(f_values, dtype=np.float32)[rng.integers(0, len(f_values), n_atoms)]
    pos, frames = brownian_frames(rng, base, n_frames, sigma, keep)
    return Trajectory(pos, f, cubic_box(L), frames, n_frames, sigma)


def fcc_crystal(seed: int, cells: int, a: float, thermal: float, vacancy: float,
                f_values: Sequence[float], n_frames: int, sigma: float, keep=None) -> Trajectory:
    rng = np.random.default_rng(seed)
    sites = fcc_sites(cells, a)
    if thermal > 0:
        sites = sites + rng.standard_normal(sites.shape) * thermal
    if vacancy > 0:
        n_keep = int(round(sites.shape[0] * (1.0 - vacancy)))
        idx = np.sort(rng.permutation(sites.shape[0])[:n_keep])
        sites = sites[idx]
    n = sites.shape[0]
    if len(f_values) == 1:
        f = np.full(n, f_values[0], dtype=np.float32)
    else:
        f = np.where(rng.random(n) < 0.5, f_values[0], f_values[1]).astype(np.float32)
    pos, frames = brownian_frames(rng, sites, n_frames, sigma, keep)
    return Trajectory(pos, f, cubic_box(cells * a), frames, n_frames, sigma)


# ----------------------------------------------------------------------------
# delay and window lists
# ----------------------------------------------------------------------------

def log_delays(T: int, n: int = 64) -> np.ndarray:
    """Strictly increasing integer delays 1 <= tau <= T-1, about log-spaced.

    tau_0 = 1, tau_k = max(tau_{k-1} + 1, round((T-1)^(k/(n-1)))); stops early
    when the list would pass T-1.
    """
    if T < 2:
        return np.zeros(0, dtype=np.int32)
    out = [1]
    for k in range(1, n):
        v = max(out[-1] + 1, int(round((T - 1) ** (k / (n - 1)))))
        if v > T - 1:
            break
        out.append(v)
    return np.asarray(out, dtype=np.int32)


def window_list_125(T: int) -> np.ndarray:
    """Window lengths K in the 1-2-5 sequence up to T."""
    out = []
    dec = 1
    while dec <= T:
        for m in (1, 2, 5):
            if m * dec <= T:
                out.append(m * dec)
        dec *= 10
    return np.asarray(sorted(set(out)), dtype=np.int32)


def rings_for_plane(grid: QGrid) -> int:
    """Number of unit-width |n| rings that cover every pixel of a plane grid."""
    m = grid.miller().astype(np.float64)
    return int(math.floor(np.sqrt((m ** 2).sum(axis=1)).max() + 0.5))


# ----------------------------------------------------------------------------
# the named workloads (sizes of the direct-method configurations)
# ----------------------------------------------------------------------------

def config0(keep=None) -> tuple[Trajectory, QGrid]:
    """4,000 atoms uniform in a 40 A box, f = 1, 10 Brownian frames
    (sigma = 0.1 A per component), 64 x 64 plane at n_z = 0."""
    traj = brownian_gas(SEED_BASE + 0, 4000, 40.0, 10, 0.1, (1.0,), keep)
    return traj, centered_plane(64)


def config1(keep=None, n_frames: int = 1000) -> tuple[Trajectory, QGrid]:
    """256,000-atom FCC crystal (a = 4 A, L = 160 A), thermal sigma 0.15 A,
    f in {1.0, 0.6} 50/50, 1,000 Brownian frames of sigma 0.05 A, 128^2 plane."""
    traj = fcc_crystal(SEED_BASE + 1, 40, 4.0, 0.15, 0.0, (1.0, 0.6), n_frames, 0.05, keep)
    return traj, centered_plane(128)


def config3() -> tuple[Trajectory, np.ndarray, QGrid]:
    """100,000 atoms uniform in a 120 A box (f = 1), one frame, 256^2 plane.

    Returns (trajectory, target positions, grid); the target speckle is the
    intensity of the positions displaced by N(0, 0.3^2) per component."""
    rng = np.random.default_rng(SEED_BASE + 3)
    L = 120.0
    base = rng.random((100_000, 3)) * L
    target = base + rng.standard_normal(base.shape) * 0.3
    f = np.ones(base.shape[0], dtype=np.float32)
    traj = Trajectory(base.astype(np.float32)[None], f, cubic_box(L), np.array([0]), 1, 0.0)
    return traj, target.astype(np.float32)[None], centered_plane(256)


def config4(keep=None, n_frames: int = 10_000) -> tuple[Trajectory, QGrid]:
    """FCC crystal of 100^3 cells (a = 4 A, L = 400 A, 4,000,000 sites) with 20 %
    vacancies (3,200,000 atoms), thermal sigma 0.2 A, f = 1, 10,000 Brownian
    frames of sigma 0.02 A, 512^2 plane (the volume mode uses
    centered_volume(128)).  `keep` selects the frames to materialise: all
    10,000 would be 384 GB of positions."""
    traj = fcc_crystal(SEED_BASE + 4, 100, 4.0, 0.2, 0.2, (1.0,), n_frames, 0.02, keep)
    return traj, centered_plane(512)


def config2_params(n_traj: int = 64, seed: int = SEED_BASE + 2) -> list[dict]:
    """Per-trajectory parameters of the batched ideal-gas workload: atom
    counts log-uniform in [2e3, 5e5], density 0.02 A^-3, frame counts uniform
    in [100, 2000], D uniform in [0.01, 1] A^2/frame, plane side in
    {64, 128, 192, 256}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_traj):
        n = int(round(math.exp(rng.uniform(math.log(2e3), math.log(5e5)))))
        T = int(rng.integers(100, 2001))
        D = float(rng.uniform(0.01, 1.0))
        side = int(rng.choice([64, 128, 192, 256]))
        out.append(dict(n_atoms=n, L=(n / 0.02) ** (1.0 / 3.0), n_frames=T, D=D,
                        sigma=math.sqrt(2.0 * D), side=side, seed=seed * 1000 + i))
    return out


def weights_inverse_q2(grid: QGrid, box: np.ndarray) -> np.ndarray:
    """Loss weights w_q = 1 / (1 + |q|^2) on a cubic-box grid, float32 [P].

    This is part of the synthetic fitting workload (the loss is the caller's),
    not of the method; |q| uses q = 2 pi n / L."""
    L = float(box[0, 0])
    m = grid.miller().astype(np.float64) * (2.0 * math.pi / L)
    return (1.0 / (1.0 + (m ** 2).sum(axis=1))).astype(np.float32)


def gas_on_device(params: dict, device, dtype_f=None):
    """One ideal-gas trajectory of `config2_params` drawn on a CUDA device with
    a seeded torch generator (the full batched workload is 75 GB of
    positions, too much to draw on the host): base positions uniform in
    [0, L)^3, then Brownian steps of sigma per component, accumulated in
    float32.  Returns (pos float32 [T][N][3], f = 1 float32 [N], box)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(params["seed"]))
    N, T, L = int(params["n_atoms"]), int(params["n_frames"]), float(params["L"])
    pos = torch.empty((T, N, 3), dtype=torch.float32, device=device)
    pos[0] = torch.rand((N, 3), generator=g, device=device, dtype=torch.float32) * L
    if T > 1:
        pos[1:] = torch.randn((T - 1, N, 3), generator=g, device=device, dtype=torch.float32) * params["sigma"]
    pos.cumsum_(0)
    f = torch.ones(N, dtype=torch.float32, device=device)
    return pos, f, cubic_box(L)


def speckle_amplitudes(seed: int, T: int, rho, device):
    """The circular complex Gaussian AR(1) amplitude a(t) = rho a(t-1) +
    sqrt(1 - rho^2) xi(t), E|a|^2 = 1, per pixel `rho` (float32 tensor [P]),
    as float32 [T][P][2] (re, im) on `device`; its normalised intermediate
    scattering function is rho^tau."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rho = rho.to(device=device, dtype=torch.float32)
    P = rho.shape[0]
    s = torch.sqrt(1.0 - rho * rho)
    out = torch.empty((T, P, 2), dtype=torch.float32, device=device)
    a = torch.complex(torch.randn(P, generator=g, device=device), torch.randn(P, generator=g, device=device))
    a = a * (0.5 ** 0.5)
    for t in range(T):
        if t > 0:
            xi = torch.complex(torch.randn(P, generator=g, device=device), torch.randn(P, generator=g, device=device))
            a = rho * a + s * xi * (0.5 ** 0.5)
        out[t, :, 0] = a.real
        out[t, :, 1] = a.imag
    return out


def speckle_series(seed: int, T: int, rho, device):
    """Synthetic speckle intensities I(t, p) = |a(t, p)|^2 of a circular complex
    Gaussian AR(1) amplitude a(t) = rho a(t-1) + sqrt(1 - rho^2) xi(t) with
    E|a|^2 = 1, per pixel correlation `rho` (float32 tensor [P] on `device`).
    Drawn on the device with a seeded torch generator; float32 [T][P].
    For this process <I(t) I(t+tau)> / <I>^2 = 1 + rho^(2 tau)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rho = rho.to(device=device, dtype=torch.float32)
    P = rho.shape[0]
    s = torch.sqrt(1.0 - rho * rho)
    out = torch.empty((T, P), dtype=torch.float32, device=device)
    a = torch.complex(torch.randn(P, generator=g, device=device), torch.randn(P, generator=g, device=device))
    a = a * (0.5 ** 0.5)
    for t in range(T):
        if t > 0:
            xi = torch.complex(torch.randn(P, generator=g, device=device), torch.randn(P, generator=g, device=device))
            a = rho * a + s * xi * (0.5 ** 0.5)
        out[t] = a.real * a.real + a.imag * a.imag
    return out
