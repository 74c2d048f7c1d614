"""Shared helpers for the GPU parity tests (error metrics and setup)."""
import numpy as np


def e_I(I, ref, miller):
    """max over frames of ||I_t - ref_t||_2 / ||ref_t||_2 over q != 0 pixels,
    and the largest relative error of the q = 0 pixel (reported apart because
    (sum f)^2 dominates any norm)."""
    I = np.asarray(I, dtype=np.float64).reshape(ref.shape)
    nz = np.any(np.asarray(miller) != 0, axis=1)
    err = 0.0
    for t in range(ref.shape[0]):
        d = np.linalg.norm(I[t, nz] - ref[t, nz])
        r = np.linalg.norm(ref[t, nz])
        err = max(err, d / r if r > 0 else d)
    z = ~nz
    e0 = 0.0
    if z.any():
        e0 = float(np.max(np.abs(I[:, z] - ref[:, z]) / np.maximum(np.abs(ref[:, z]), 1e-300)))
    return err, e0


def amp_err(A, ref):
    """||A - ref|| / ||ref|| over all entries (complex)."""
    A = np.asarray(A, dtype=np.float64)
    a = A[..., 0] + 1j * A[..., 1]
    a = a.reshape(ref.shape)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
