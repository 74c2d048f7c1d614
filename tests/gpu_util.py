"""Shared helpers for the GPU parity tests (error metrics and setup).

Two kinds of intensity metric are asserted together:
  * e_I, norm-wise: max over frames of ||I_t - ref_t||_2 / ||ref_t||_2 over the
    q != 0 pixels, with the q = 0 pixel's relative error apart;
  * e_pix, element-wise: max over frames and q != 0 pixels of
    |I - ref| / max(ref, mean_t(ref)).  On pixels darker than the frame's mean
    intensity this is |dI| / mean(I_ref); on brighter ones (bright speckles,
    Bragg peaks) it is the pixel's relative error.  A single wrong pixel -- a
    tile seam, a mirror line, a lost piece of a split unit -- is off by about
    the mean intensity and fails it, while e_I over 16,384 pixels would let it
    pass.
The element-wise bounds (PIX_TOL) come from the largest values measured on
the workloads of the tests: 6.5e-4 on the split paths (the 256,000-atom
crystal at frame 0, whose diffuse amplitudes are four times smaller than the
4,096-atom chunk sums that carry the FP32 accumulation error) and 7.2e-7 on
the FP32 path; the bounds leave a factor of three and seven.
"""
import numpy as np

NORM_TOL = {"fp32": 1e-6, "fp32f": 1e-6, "fp16": 1e-4, "bf16": 1e-4}
PIX_TOL = {"fp32": 5e-6, "fp32f": 5e-6, "fp16": 2e-3, "bf16": 2e-3}


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


def e_pix(I, ref, miller):
    """Element-wise error: max over frames and q != 0 pixels of
    |I - ref| / max(ref, mean over the frame's q != 0 pixels of ref)."""
    I = np.asarray(I, dtype=np.float64).reshape(ref.shape)
    nz = np.any(np.asarray(miller) != 0, axis=1)
    err = 0.0
    for t in range(ref.shape[0]):
        r = ref[t, nz]
        if r.size == 0:
            continue
        mean = float(np.mean(r))
        den = np.maximum(r, mean)
        d = np.abs(I[t, nz] - r)
        if mean <= 0.0:
            err = max(err, float(d.max()))
            continue
        err = max(err, float(np.max(d / den)))
    return err


def mean_dev(I, ref, miller):
    """max over frames of max |I - ref| / mean(ref) over q != 0 pixels (the
    plain mean-normalised deviation; reported, bounded where no Bragg peak
    dominates)."""
    I = np.asarray(I, dtype=np.float64).reshape(ref.shape)
    nz = np.any(np.asarray(miller) != 0, axis=1)
    err = 0.0
    for t in range(ref.shape[0]):
        r = ref[t, nz]
        if r.size == 0 or np.mean(r) <= 0:
            continue
        err = max(err, float(np.max(np.abs(I[t, nz] - r)) / np.mean(r)))
    return err


def check_I(I, ref, miller, prec, norm_tol=None, pix_tol=None, what=""):
    """Assert e_I, the q = 0 error and e_pix within the tolerances of `prec`;
    returns (e_I, e0, e_pix)."""
    nt = NORM_TOL[prec] if norm_tol is None else norm_tol
    pt = PIX_TOL[prec] if pix_tol is None else pix_tol
    e, e0 = e_I(I, ref, miller)
    ep = e_pix(I, ref, miller)
    assert e <= nt, (what, prec, "e_I", e)
    assert e0 <= nt, (what, prec, "q=0", e0)
    assert ep <= pt, (what, prec, "e_pix", ep)
    return e, e0, ep


def amp_err(A, ref):
    """||A - ref|| / ||ref|| over all entries (complex)."""
    A = np.asarray(A, dtype=np.float64)
    a = A[..., 0] + 1j * A[..., 1]
    a = a.reshape(ref.shape)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def amp_pix(A, ref):
    """Element-wise amplitude error: max over entries of
    |A - ref| / max(|ref|, rms of ref over the frame); the last axis of `ref`
    is the pixel axis."""
    A = np.asarray(A, dtype=np.float64)
    a = (A[..., 0] + 1j * A[..., 1]).reshape(ref.shape)
    ref2 = ref.reshape(-1, ref.shape[-1])
    a2 = a.reshape(ref2.shape)
    rms = np.sqrt(np.mean(np.abs(ref2) ** 2, axis=1, keepdims=True))
    den = np.maximum(np.abs(ref2), rms)
    return float(np.max(np.abs(a2 - ref2) / np.where(den > 0, den, 1.0)))
