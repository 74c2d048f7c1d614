"""Element-wise parity where defects of the tensor-core path would hide
(Sec. 2.2 Eq. Iq_pq; Sec. 3.1, Algorithm 1 in factorised form), on the
256,000-atom / 1,000-frame FCC workload at full size.

A defect at a seam moves single pixels or lines by about the mean intensity:
a norm over 16,384 pixels barely sees it, so these tests compare every
checked pixel's intensity (e_pix) and complex amplitude (amp_pix) with the
FP64 oracle:
  * the centred 128^2 plane of the bench: the lines where the centred tile's
    slots change (n = -64, -33/-32/-31, -1/0/1, 31/32, 63 on either axis),
    the Bragg reflections of the plane, and frames on both sides of the
    first split unit of the last wave (for 74 and for 76 CTA pairs) and the
    last frame;
  * a grid of 2 x 3 ragged tiles on two planes (n_z = 0, 1): the rows and
    columns 0, 127, 128, 255 (and the ragged last column block) of every
    tile;
  * a centred 192^2 plane contracted as a half plus its mirror, and an 81^3
    volume contracted as its planes n_z <= 0: the mirror lines n_x = 0, +-1
    and the planes n_z = 0, +-1, where the conjugation of mirrored
    amplitudes shows.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import amp_err, amp_pix, check_I
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


@pytest.fixture(scope="module")
def crystal(xs):
    traj, grid = wl.config1()
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    yield traj, grid, p, fd
    del p, fd
    torch.cuda.empty_cache()


def _check(xs, traj, I, A, grid, frames, pick, what):
    m = grid.miller()
    T = I.shape[0]
    ref = oracle.amplitude(traj.pos[frames], traj.f, traj.box, m[pick])
    got_I = I.reshape(T, -1)[frames][:, pick].cpu().numpy()
    got_A = A.reshape(T, -1, 2)[frames][:, pick].cpu().numpy()
    check_I(got_I, np.abs(ref) ** 2, m[pick], "fp16", what=what)
    assert amp_err(got_A, ref) <= 1e-4, what
    ap = amp_pix(got_A, ref)
    assert ap <= 2e-3, (what, ap)


def test_centred_plane_slot_lines_peaks_and_split_pieces(xs, crystal):
    traj, grid, p, fd = crystal
    I, A = xs.intensity(p, fd, traj.box, grid, "fp16", want_amp=True)
    xs.Context.get().sync_status()
    m = grid.miller()
    lines = np.array([-64, -63, -33, -32, -31, -1, 0, 1, 31, 32, 63])
    on_line = np.isin(m[:, 0], lines) | np.isin(m[:, 1], lines)
    bragg = np.all(m % 40 == 0, axis=1)
    pick = np.flatnonzero(on_line | bragg)
    # 1,000 units on 74 pairs: frames 962.. are split along the atoms; on 76
    # pairs frames 988..
    frames = [0, 961, 962, 987, 988, 999]
    _check(xs, traj, I, A, grid, frames, pick, "centred 128^2")
    # every frame is finite and the mirrored slots hold conjugate pairs
    assert torch.isfinite(I).all()


def test_multi_tile_grid_rows_127_128(xs, crystal):
    traj, _, p, fd = crystal
    grid = wl.QGrid(-100, 256, -130, 300, 0, 2)
    I, A = xs.intensity(p, fd, traj.box, grid, "fp16", want_amp=True)
    xs.Context.get().sync_status()
    m = grid.miller()
    lx, ly = m[:, 0] - grid.nx0, m[:, 1] - grid.ny0
    pick = np.flatnonzero(np.isin(lx, [0, 127, 128, 255]) | np.isin(ly, [0, 127, 128, 255, 256, 299]))
    _check(xs, traj, I, A, grid, [0, 500, 999], pick, "2 x 3 tiles x 2 planes")
    del I, A


def test_half_grid_mirror_lines(xs, crystal):
    traj, _, p, fd = crystal
    rng = np.random.default_rng(44)
    plane = wl.centered_plane(192)
    I, A = xs.intensity(p, fd, traj.box, plane, "fp16", want_amp=True)
    xs.Context.get().sync_status()
    m = plane.miller()
    pick = np.flatnonzero(np.isin(m[:, 0], [-96, -1, 0, 1, 95]) | np.isin(m[:, 1], [-96, 0, 95]))
    _check(xs, traj, I, A, plane, [0, 999], pick, "192^2 half plane")
    del I, A
    vol = wl.QGrid(-40, 81, -40, 81, -40, 81)
    Iv, Av = xs.intensity(p[:40].contiguous(), fd, traj.box, vol, "fp16", want_amp=True)
    xs.Context.get().sync_status()
    m = vol.miller()
    parts = []
    for nz in (-40, -1, 0, 1, 40):
        sel = np.flatnonzero(m[:, 2] == nz)
        line = sel[np.isin(m[sel, 0], [-1, 0, 1])]
        parts += [line, rng.choice(sel, 300, replace=False)]
    pick = np.unique(np.concatenate(parts))
    _check(xs, traj, Iv, Av, vol, [0, 39], pick, "81^3 volume, planes n_z <= 0 contracted")
