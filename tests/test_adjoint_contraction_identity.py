"""The identity the tensor-core adjoint is built on, checked in float64 on the
CPU against the oracle's analytic gradient (no CUDA code is involved).

For q on the reciprocal lattice the phase factorises (Sec. 3.1), so with
H_q = dL/dI_q conj(S_q), rows q = (n_x, n_z) and the column index n_y:
  Z(q, j) = sum_y H(q, y) E_y(y, j),  Z_y(q, j) = sum_y n_y H(q, y) E_y(y, j).
The kernel computes these as one real contraction with the complex parts
folded into K (k' = 2y + p): the rows [Re H, -Im H] and [Im H, Re H] (and n_y
times them) against B[j][2y + p] = (Re E_y, Im E_y) give Re Z, Im Z, Re Z_y
and Im Z_y.  Per atom, Im T = sum_q (n_x, 1, n_z) Im[E_xz Z or Z_y] and
dL/dr = -4 pi f h^-T Im T.  A sign, a transposed h or a swapped real and
imaginary part anywhere in this chain fails the comparison."""
import numpy as np
import pytest

import oracle


def _folded_gradient(pos, f, box, grid, G):
    nx0, nx, ny0, ny, nz0, nz = grid
    hinv = np.linalg.inv(box)
    s = pos @ hinv.T                                   # fractional coordinates
    mx, my, mz = np.meshgrid(np.arange(nx0, nx0 + nx), np.arange(ny0, ny0 + ny), np.arange(nz0, nz0 + nz),
                             indexing="ij")
    miller = np.stack([mx.transpose(2, 1, 0).ravel(), my.transpose(2, 1, 0).ravel(),
                       mz.transpose(2, 1, 0).ravel()], axis=1)   # [nz][ny][nx], n_x fastest
    S = oracle.amplitude(pos[None], f, box, miller)[0]
    H = (G * np.conj(S)).reshape(nz, ny, nx)
    nyv = np.arange(ny0, ny0 + ny, dtype=np.float64)
    Ey = np.exp(2j * np.pi * np.outer(nyv, s[:, 1]))   # [y][atom]
    # B[j][2y + p]: real and imaginary parts interleaved along K
    B = np.empty((pos.shape[0], 2 * ny))
    B[:, 0::2] = Ey.real.T
    B[:, 1::2] = Ey.imag.T
    T = np.zeros((pos.shape[0], 3))
    for z in range(nz):
        for x in range(nx):
            h = H[z, :, x]
            rows = np.empty((4, 2 * ny))
            rows[0, 0::2], rows[0, 1::2] = h.real, -h.imag    # -> Re Z
            rows[1, 0::2], rows[1, 1::2] = h.imag, h.real     # -> Im Z
            rows[2] = rows[0] * np.repeat(nyv, 2)             # -> Re Z_y
            rows[3] = rows[1] * np.repeat(nyv, 2)             # -> Im Z_y
            D = rows @ B.T                                     # [4][atom]
            n_x, n_z = nx0 + x, nz0 + z
            E = np.exp(2j * np.pi * (n_x * s[:, 0] + n_z * s[:, 2]))
            im_z = E.imag * D[0] + E.real * D[1]              # Im[E Z]
            im_zy = E.imag * D[2] + E.real * D[3]             # Im[E Z_y]
            T[:, 0] += n_x * im_z
            T[:, 1] += im_zy
            T[:, 2] += n_z * im_z
    grad = -4.0 * np.pi * f[:, None] * (T @ hinv)            # (h^-T v)_c = sum_b hinv[b][c] v_b
    return grad, miller, S


@pytest.mark.parametrize("grid,cell", [
    ((-9, 18, -7, 15, 0, 1), np.eye(3) * 17.0),                                      # plane at n_z = 0
    ((-4, 9, -5, 11, -2, 4), np.array([[14.0, 2.0, 0.0], [0.0, 12.0, 1.5], [-1.0, 0.0, 11.0]])),  # triclinic volume
])
def test_folded_contraction_equals_analytic_gradient(grid, cell):
    rng = np.random.default_rng(17)
    N = 120
    pos = (rng.random((N, 3)) @ cell.T).astype(np.float32).astype(np.float64)
    f = rng.uniform(0.5, 1.5, N)
    nx, ny, nz = grid[1], grid[3], grid[5]
    G = rng.standard_normal(nx * ny * nz)
    got, miller, S = _folded_gradient(pos, f, cell, grid, G)
    ref = oracle.grad_analytic(pos, f, cell, miller, G, amp=S)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11
