"""Pins of the oracle's Ewald-sphere detector slice (arXiv 2204.13241 Fig. 5:
the speckle on the spherical slice |k_f| = |k_i|, k_f = k_i + q):
  * cubic box, beam along z: the near root has the closed form
    n_z = (L / 2 pi) (sqrt(k^2 - q_perp^2) - k), and the chosen n_z is the
    integer of the near half-chord closest to the sphere (brute-force scan);
  * q = 0 is on the sphere; lines with q_perp > k miss it;
  * a triclinic cell and a tilted beam: every point lies within half a lattice
    step (along n_z) of the sphere."""
import math

import numpy as np

import oracle


def test_cubic_beam_along_z_closed_form_and_brute_force():
    L, lam = 40.0, 1.3
    k = 2 * math.pi / lam
    box = np.eye(3) * L
    m, valid = oracle.ewald_points(box, [0.0, 0.0, k], -40, 80, -36, 72)
    qx = 2 * math.pi * m[:, 0] / L
    qy = 2 * math.pi * m[:, 1] / L
    qp2 = qx * qx + qy * qy
    assert np.array_equal(valid, qp2 <= k * k)
    dz = 2 * math.pi / L
    for i in np.flatnonzero(valid)[::7]:
        root = (math.sqrt(k * k - qp2[i]) - k) / dz
        assert math.floor(root) <= m[i, 2] <= math.ceil(root)
        # brute force over the near half-chord n in [vertex, 0]
        best, bd = None, None
        for n in range(int(math.floor(-k / dz)) - 1, 1):
            d = abs(math.sqrt(qp2[i] + (n * dz + k) ** 2) - k)
            if bd is None or d < bd - 1e-15 or (abs(d - bd) <= 1e-15 and abs(n) < abs(best)):
                best, bd = n, d
        assert m[i, 2] == best, (m[i], best)
    zero = np.flatnonzero((m[:, 0] == 0) & (m[:, 1] == 0))
    assert valid[zero].all() and m[zero, 2][0] == 0


def test_triclinic_cell_tilted_beam_points_near_sphere():
    h = np.array([[30.0, 4.0, -2.0], [0.0, 27.0, 3.0], [0.0, 0.0, 33.0]])
    k = np.array([0.3, -0.2, 8.0])
    m, valid = oracle.ewald_points(h, k, -20, 40, -24, 48)
    Ht = 2 * math.pi * np.linalg.inv(h).T
    q = m.astype(np.float64) @ Ht.T
    dist = np.abs(np.linalg.norm(q + k, axis=1) - np.linalg.norm(k))
    step = np.linalg.norm(Ht[:, 2])
    assert valid.sum() > 0.9 * valid.size
    assert np.all(dist[valid] <= 0.5 * step + 1e-12)
    # moving one step along n_z never brings the point closer to the sphere
    for dn in (-1, 1):
        q2 = (m + np.array([0, 0, dn])).astype(np.float64) @ Ht.T
        d2 = np.abs(np.linalg.norm(q2 + k, axis=1) - np.linalg.norm(k))
        assert np.all(dist[valid] <= d2[valid] + 1e-12)
