"""Parity of the CUDA intensity paths with the FP64 oracle (Sec. 3.1,
Algorithm 1): the plain FP32 direct kernel at <= 1e-6 and the split FP16 /
BF16 tensor-core kernel at <= 1e-4 (e_I, relative L2 over q != 0 pixels per
frame), each also element-wise (e_pix, |dI| / max(I_ref, mean I_ref) per
pixel, see gpu_util), on ragged small shapes, edge cases, the tile seams,
centred-tile slot boundaries and split pieces of the full 256,000-atom /
1,000-frame / 128^2 workload, and sampled frames of that workload."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_util import NORM_TOL as TOL, PIX_TOL as PIX, amp_err, amp_pix, check_I, e_I, e_pix
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


def _run(xs, pos, f, box, grid, prec, amp=False):
    p = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    fd = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    out = xs.intensity(p, fd, box, grid, prec, want_amp=amp)
    xs.Context.get().sync_status()
    if amp:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


def _case(seed, N, T, L, sigma=0.2, f_mixed=True):
    rng = np.random.default_rng(seed)
    base = rng.random((N, 3)) * L
    steps = rng.standard_normal((T, N, 3)) * sigma
    steps[0] = 0
    pos = (base[None] + np.cumsum(steps, axis=0)).astype(np.float32)
    f = np.where(rng.random(N) < 0.5, 1.0, 0.6).astype(np.float32) if f_mixed else np.ones(N, np.float32)
    return pos, f, np.eye(3) * L


@pytest.mark.parametrize("prec", ["fp32", "fp32f"])
def test_fp32_direct_config0_full(xs, prec):
    traj, grid = wl.config0()
    I = _run(xs, traj.pos, traj.f, traj.box, grid, prec)
    ref = oracle.intensity(traj.pos, traj.f, traj.box, grid.miller())
    check_I(I, ref, grid.miller(), prec)


def test_factored_fp32_at_the_adjoint_workload_size(xs):
    # 100,000 atoms, 256^2 plane: the forward of the fitting workload, against
    # the oracle on sampled pixels (q = 0 included)
    traj, _, grid = wl.config3()
    I = _run(xs, traj.pos, traj.f, traj.box, grid, "fp32f").reshape(1, -1)
    m = grid.miller()
    rng = np.random.default_rng(31)
    pick = np.unique(np.concatenate([np.flatnonzero(np.all(m == 0, axis=1)), rng.choice(m.shape[0], 2048, replace=False)]))
    ref = oracle.intensity(traj.pos, traj.f, traj.box, m[pick])
    check_I(I[:, pick], ref, m[pick], "fp32f")


@pytest.mark.parametrize("prec", ["fp32", "fp32f", "fp16", "bf16"])
@pytest.mark.parametrize("N,T,grid", [
    (1000, 3, wl.QGrid(-48, 96, -40, 80, 0, 1)),      # ragged atoms and tiles
    (64, 2, wl.QGrid(-64, 128, -64, 128, 1, 1)),      # exact tiles, q_z != 0
    (333, 2, wl.QGrid(-5, 11, -7, 13, -2, 5)),        # small volume
    (4097, 1, wl.QGrid(0, 200, -100, 260, 0, 1)),     # several x and y tiles
])
def test_ragged_shapes(xs, prec, N, T, grid):
    pos, f, box = _case(7 + N, N, T, 23.0)
    I = _run(xs, pos, f, box, grid, prec)
    ref = oracle.intensity(pos, f, box, grid.miller())
    check_I(I, ref, grid.miller(), prec)


@pytest.mark.parametrize("prec", ["fp32", "fp32f", "fp16"])
def test_amplitude_matches_oracle(xs, prec):
    pos, f, box = _case(3, 700, 2, 17.0)
    grid = wl.QGrid(-20, 40, -20, 40, 0, 1)
    I, A = _run(xs, pos, f, box, grid, prec, amp=True)
    ref = oracle.amplitude(pos, f, box, grid.miller())
    assert amp_err(A, ref) <= TOL[prec]
    assert amp_pix(A, ref) <= PIX[prec]
    check_I(I.reshape(2, -1), np.abs(ref) ** 2, grid.miller(), prec)
    assert np.allclose(I.reshape(-1), (A[..., 0] ** 2 + A[..., 1] ** 2).reshape(-1), rtol=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "fp32f", "fp16", "bf16"])
def test_triclinic_cell(xs, prec):
    rng = np.random.default_rng(5)
    h = np.array([[12.0, 3.0, -1.5], [0.0, 10.0, 2.5], [1.0, 0.0, 9.0]])
    s = rng.random((500, 3))
    pos = (s @ h.T).astype(np.float32)[None]
    f = rng.uniform(0.5, 1.5, 500).astype(np.float32)
    grid = wl.QGrid(-10, 20, -9, 18, -1, 3)
    I = _run(xs, pos, f, h, grid, prec)
    ref = oracle.intensity(pos, f, h, grid.miller())
    check_I(I, ref, grid.miller(), prec)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_symmetric_volume_from_half_and_mirrors(xs, prec):
    # n in [-6, 6]^3 maps onto itself under n -> -n: the tensor path contracts
    # the planes n_z <= 0 and reads the others from their mirrors, using
    # S(-q) = conj S(q) for real form factors; the amplitude checks the
    # conjugation
    pos, f, box = _case(31, 900, 2, 19.0)
    grid = wl.QGrid(-6, 13, -6, 13, -6, 13)
    I, A = _run(xs, pos, f, box, grid, prec, amp=True)
    ref = oracle.amplitude(pos, f, box, grid.miller())
    assert amp_err(A, ref) <= TOL[prec]
    assert amp_pix(A, ref) <= PIX[prec]
    check_I(I.reshape(2, -1), np.abs(ref) ** 2, grid.miller(), prec)


@pytest.mark.parametrize("grid", [
    wl.QGrid(-40, 81, -40, 81, -40, 81),   # the 81^3 grid of the paper's Table 1: 41 planes contracted
    wl.centered_plane(192),                # two tiles instead of four
])
def test_half_grid_against_oracle(xs, grid):
    rng = np.random.default_rng(33)
    N, L = 4000, 59.19
    pos = (rng.random((1, N, 3)) * L).astype(np.float32)
    f = np.ones(N, np.float32)
    box = np.eye(3) * L
    I = _run(xs, pos, f, box, grid, "fp16").reshape(1, -1)
    m = grid.miller()
    pick = np.unique(np.concatenate([np.flatnonzero(np.all(m == 0, axis=1)),
                                     np.flatnonzero((m[:, 0] == 1) | (m[:, 2] == 1))[:2000],
                                     rng.choice(m.shape[0], 3000, replace=False)]))
    ref = oracle.intensity(pos, f, box, m[pick])
    check_I(I[:, pick], ref, m[pick], "fp16")


@pytest.mark.parametrize("prec", ["fp32", "fp32f", "fp16", "bf16"])
def test_edge_cases_single_and_zero_atoms(xs, prec):
    grid = wl.QGrid(-8, 16, -8, 16, 0, 1)
    box = np.eye(3) * 9.0
    one = np.array([[[1.25, -3.5, 7.0]]], dtype=np.float32)
    I = _run(xs, one, np.array([0.7], np.float32), box, grid, prec)
    assert np.allclose(I, 0.49, rtol=TOL[prec] * 4)
    empty = np.zeros((2, 0, 3), np.float32)
    p = torch.zeros((2, 0, 3), dtype=torch.float32, device="cuda")
    fz = torch.zeros((0,), dtype=torch.float32, device="cuda")
    out = xs.intensity(p, fz, box, grid, prec)
    assert torch.count_nonzero(out).item() == 0
    del empty


def test_host_streamed_positions_match_device(xs):
    pos, f, box = _case(11, 2000, 6, 21.0)
    grid = wl.QGrid(-32, 64, -32, 64, 0, 1)
    dev = _run(xs, pos, f, box, grid, "fp16")
    hp = torch.from_numpy(pos).pin_memory()
    hf = torch.from_numpy(f).pin_memory()
    host_out = xs.intensity(hp, hf, box, grid, "fp16")
    assert not host_out.is_cuda
    assert np.array_equal(host_out.numpy(), dev)


def _host_run(xs, pos, f, box, grid, shift, pinned):
    pbuf = torch.empty(pos.size + shift, dtype=torch.float32)
    fbuf = torch.empty(f.size + 3 - shift, dtype=torch.float32)
    if pinned:
        pbuf, fbuf = pbuf.pin_memory(), fbuf.pin_memory()
    hp = pbuf[shift:].view(pos.shape)
    hf = fbuf[3 - shift:]
    hp.copy_(torch.from_numpy(pos))
    hf.copy_(torch.from_numpy(f))
    assert hp.is_pinned() == pinned
    out = torch.empty((pos.shape[0], 1, grid.ny, grid.nx), dtype=torch.float32, device="cuda")
    xs.intensity(hp, hf, box, grid, "fp16", out=out)
    xs.Context.get().sync_status()
    return out.cpu().numpy()


@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_host_positions_at_any_alignment_pinned_or_pageable(xs, shift):
    # host positions and form factors, page-locked or pageable, starting at
    # any float offset, give the same bits; 40,000 atoms over 300 frames make
    # two chunks, whose launches split the work differently from one launch
    # over all frames, so the device-resident result is met within the
    # tolerance instead
    pos, f, box = _case(17, 40000, 300, 70.0)
    grid = wl.QGrid(-16, 32, -16, 32, 0, 1)
    ref = _host_run(xs, pos, f, box, grid, 0, False)
    got = _host_run(xs, pos, f, box, grid, shift, True)
    assert np.array_equal(got, ref)
    if shift:
        assert np.array_equal(_host_run(xs, pos, f, box, grid, shift, False), ref)
    dev = _run(xs, pos, f, box, grid, "fp16")
    m = grid.miller()
    err, err0 = e_I(got.reshape(300, -1), dev.reshape(300, -1).astype(np.float64), m)
    assert err <= 1e-4 and err0 <= 1e-4, (err, err0)


def test_host_streaming_over_several_chunks(xs):
    # 64,000 atoms are 768 kB per frame: host positions are streamed in chunks
    # that start near 64 MB (87 frames) and double, so 200 frames take two
    # chunks with their own launches; the output goes to host memory too
    pos, f, box = _case(13, 64000, 200, 90.0, f_mixed=False)
    grid = wl.QGrid(-32, 64, -32, 64, 0, 1)
    dev = _run(xs, pos, f, box, grid, "fp16")
    hp = torch.from_numpy(pos).pin_memory()
    hf = torch.from_numpy(f).pin_memory()
    host_out = xs.intensity(hp, hf, box, grid, "fp16").numpy().reshape(200, -1)
    m = grid.miller()
    err, err0 = e_I(host_out, dev.reshape(200, -1), m)
    assert err <= 1e-4 and err0 <= 1e-6, (err, err0)
    assert e_pix(host_out, dev.reshape(200, -1).astype(np.float64), m) <= 2e-3
    pix = np.random.default_rng(3).choice(m.shape[0], 48, replace=False)
    for t in (0, 86, 87, 199):  # both sides of the chunk boundary
        ref = oracle.intensity(pos[t:t + 1], f, box, m[pix])
        check_I(host_out[t:t + 1, pix], ref, m[pix], "fp16", what=f"frame {t}")


def test_nonfinite_position_is_reported(xs):
    from paper_2204_13241_gb300 import _native as nat
    pos, f, box = _case(12, 100, 1, 10.0)
    pos[0, 17, 1] = np.nan
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    xs.intensity(p, fd, box, wl.QGrid(-4, 8, -4, 8, 0, 1), "fp32")
    with pytest.raises(nat.XsError) as ei:
        xs.Context.get().sync_status()
    assert ei.value.status == 6
    xs.Context.get().sync_status()  # cleared


@pytest.mark.parametrize("prec", ["fp32", "fp32f", "fp16"])
def test_periodic_images_give_identical_records(xs, prec):
    # box 16 and positions on a 2^-8 grid: shifts by up to 2^10 boxes stay
    # exact in float32, and the turn counts rint(x 2^32 / 16) mod 2^32 of an
    # atom and of its images agree, so the intensities agree bit for bit
    rng = np.random.default_rng(21)
    N, T, L = 3000, 2, 16.0
    pos = (np.floor(rng.random((T, N, 3)) * L * 256) / 256).astype(np.float32)
    shift = rng.integers(-1024, 1025, (T, N, 3)).astype(np.float32) * np.float32(L)
    far = (pos + shift).astype(np.float32)
    assert np.array_equal(far - shift, pos)
    f = rng.uniform(0.5, 1.5, N).astype(np.float32)
    box = np.eye(3) * L
    grid = wl.QGrid(-40, 80, -40, 80, 0, 1)
    I0 = _run(xs, pos, f, box, grid, prec)
    I1 = _run(xs, far, f, box, grid, prec)
    assert np.array_equal(I0, I1)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_unwrapped_positions_far_from_the_cell(xs, prec):
    # a box that is no power of two, atoms about 1,000 and 2^17 boxes out
    # (both signs): the integer turn counts stay exact there
    rng = np.random.default_rng(22)
    N, L = 1200, 21.7
    base = rng.random((N, 3)) * L
    k = np.where(rng.random((N, 3)) < 0.5, 1000.0, 2.0 ** 17) * np.where(rng.random((N, 3)) < 0.5, 1.0, -1.0)
    pos = (base + k * L).astype(np.float32)[None]
    f = rng.uniform(0.5, 1.5, N).astype(np.float32)
    box = np.eye(3) * L
    grid = wl.QGrid(-16, 32, -16, 32, -1, 3)
    I = _run(xs, pos, f, box, grid, prec)
    ref = oracle.intensity(pos, f, box, grid.miller())
    check_I(I, ref, grid.miller(), prec)


def test_position_beyond_the_turn_range_is_reported(xs):
    # more than 2^18 cells out: rejected through the error word
    from paper_2204_13241_gb300 import _native as nat
    pos, f, box = _case(14, 300, 1, 10.0)
    pos[0, 5, 0] = np.float32(10.0 * 2.0 ** 19)
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    xs.intensity(p, fd, box, wl.QGrid(-64, 128, -64, 128, 0, 1), "fp16")
    with pytest.raises(nat.XsError) as ei:
        xs.Context.get().sync_status()
    assert ei.value.status == 6
    xs.Context.get().sync_status()  # cleared


def test_bounded_wait_timeout_is_reported_and_context_survives(xs):
    from paper_2204_13241_gb300 import _native as nat
    pos, f, box = _case(13, 4096, 4, 20.0)
    grid = wl.QGrid(-32, 64, -32, 64, 0, 1)
    ctx = xs.Context.get()
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    ctx.set_wait_timeout_ns(1)   # no producer can fill a stage within 1 ns
    try:
        xs.intensity(p, fd, box, grid, "fp16")
        with pytest.raises(nat.XsError) as ei:
            ctx.sync_status()
        assert ei.value.status == 5
    finally:
        ctx.set_wait_timeout_ns(2_000_000_000)
    I = xs.intensity(p, fd, box, grid, "fp16")
    ctx.sync_status()
    ref = oracle.intensity(pos, f, box, grid.miller())
    check_I(I.cpu().numpy(), ref, grid.miller(), "fp16")


def test_tuned_chunks_keep_parity(xs):
    pos, f, box = _case(14, 20000, 2, 30.0)
    grid = wl.QGrid(-64, 128, -64, 128, 0, 1)
    p = torch.from_numpy(pos).cuda()
    fd = torch.from_numpy(f).cuda()
    xs.tune(p, fd, box, grid, "fp16")
    I = xs.intensity(p, fd, box, grid, "fp16")
    xs.Context.get().sync_status()
    ref = oracle.intensity(pos, f, box, grid.miller())
    check_I(I.cpu().numpy(), ref, grid.miller(), "fp16")


def test_fcc_bragg_peaks_on_tensor_path(xs):
    # perfect crystal: I = N^2 at allowed reflections, 0 elsewhere (selection rules)
    cells, a = 8, 4.0
    sites = wl.fcc_sites(cells, a).astype(np.float32)[None]
    N = sites.shape[1]
    grid = wl.QGrid(-16, 32, -16, 32, 0, 1)
    for prec in ("fp16", "bf16"):
        I = _run(xs, sites, np.ones(N, np.float32), np.eye(3) * cells * a, grid, prec).reshape(-1)
        m = grid.miller()
        allowed = np.all(m % cells == 0, axis=1) & np.all(((m // cells) % 2) == ((m[:, :1] // cells) % 2), axis=1)
        assert np.allclose(I[allowed], float(N) ** 2, rtol=1e-4)
        assert np.all(I[~allowed] <= 1e-6 * N * N)


def test_config1_full_size_sampled_frames(xs):
    """256,000 atoms x 1,000 frames x 128^2 plane on the split FP16 path, in the
    bench's launch configuration; four frames checked against the oracle on a
    seeded sample of 1,024 pixels (q = 0 included)."""
    traj, grid = wl.config1()
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I = xs.intensity(p, fd, traj.box, grid, "fp16")
    xs.Context.get().sync_status()
    del p
    frames = [0, 1, 500, 999]
    rng = np.random.default_rng(99)
    m = grid.miller()
    pix = np.unique(np.concatenate([[np.flatnonzero(np.all(m == 0, axis=1))[0]],
                                    rng.choice(m.shape[0], 1024, replace=False)]))
    ref = oracle.intensity(traj.pos[frames], traj.f, traj.box, m[pix])
    got = I.reshape(I.shape[0], -1)[frames][:, pix].cpu().numpy()
    check_I(got, ref, m[pix], "fp16")
    assert torch.isfinite(I).all()
