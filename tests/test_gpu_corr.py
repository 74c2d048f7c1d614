"""Parity of the CUDA g2 (Sec. 2.3 Eq. g2_def) and XSVS contrast (Eqs.
inte_Iq, bq_Iq) with the FP64 oracle: stage parity on the same intensity
array, ragged sizes and edge cases, and the end-to-end chain of the
4,000-atom workload (FP32 intensity -> g2, contrast) at <= 1e-6."""
import numpy as np
import pytest
import torch

import oracle
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


@pytest.mark.parametrize("T,P,taus", [
    (37, 1000, [0, 1, 2, 5, 36]),
    (200, 129, list(range(0, 40))),         # more delays than one group
    (1, 5, [0]),
    (1000, 4096, list(wl.log_delays(1000))),
    # frame segments are whole 64-frame blocks, up to 8: at 577 and 1,100
    # frames the last segments hold no frame and must still add zeros
    (577, 200, [0, 1, 3, 64, 576]),
    (1100, 300, [1, 2, 3, 17, 1099]),
    (40000, 64, [0, 1, 7, 4095, 4096, 39999]),  # several 4,096-frame FP32 blocks per segment
    # the longest series kept whole for 32 pixels per block, and one frame
    # more (16 pixels per block)
    (1600, 70, [0, 1, 255, 256, 799, 1599]),
    (1601, 33, [0, 2, 256, 1600]),
    # 16 pixels per block up to 3,200 frames, then the segment kernel
    (3200, 40, [0, 1, 9, 1000, 3199]),
    (3201, 17, [0, 5, 3200]),
])
def test_g2_stage_parity(xs, T, P, taus):
    rng = np.random.default_rng(T + P)
    I = rng.exponential(50.0, (T, P)).astype(np.float32)
    g, mean = xs.g2(torch.from_numpy(I).cuda(), taus)
    xs.Context.get().sync_status()
    ref, mref = oracle.g2(I, taus)
    assert np.allclose(mean.cpu().numpy(), mref, rtol=1e-7)
    assert np.allclose(g.cpu().numpy(), ref, rtol=2e-6, atol=0)


def test_g2_rejects_bad_delay(xs):
    from paper_2204_13241_gb300 import _native as nat
    I = torch.ones((5, 3), device="cuda")
    with pytest.raises(nat.XsError):
        xs.g2(I, [5])
    with pytest.raises(nat.XsError):
        xs.g2(I, [-1])


@pytest.mark.parametrize("T,side,Ks,width", [
    (23, 24, [1, 2, 3, 7, 23], 1.0),
    (100, 50, [1, 5, 10, 33, 100], 0.5),
    (10, 64, list(range(1, 11)), 1.0),
    (700, 40, [1, 3, 7, 50, 700], 1.0),      # prefix sums over 8 frame segments
])
def test_xsvs_stage_parity(xs, T, side, Ks, width):
    rng = np.random.default_rng(T * side)
    grid = wl.centered_plane(side)
    I = rng.exponential(10.0, (T, grid.n_pixels)).astype(np.float32)
    box = np.eye(3) * 31.0
    R = wl.rings_for_plane(grid)
    beta, counts = xs.xsvs_contrast(torch.from_numpy(I).cuda(), grid, box, Ks, R, width)
    xs.Context.get().sync_status()
    rings = oracle.ring_index(box, grid.miller(), width, R)
    ref, cref = oracle.xsvs_contrast(I, Ks, rings, R)
    assert np.array_equal(counts, cref)
    b = beta.cpu().numpy()
    assert np.array_equal(np.isnan(b), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.allclose(b[ok], ref[ok], rtol=1e-9, atol=1e-12)


def test_xsvs_hand_series_through_library(xs):
    # the golden hand example laid on a 3-pixel-wide grid: pixels with |n| = 1
    # form ring 1; the values come from tests/golden/xsvs_hand.txt's ring 1
    grid = wl.QGrid(-1, 3, 0, 1, 0, 1)        # n = (-1,0,0), (0,0,0), (1,0,0)
    frames = np.array([[1.0, 99.0, 1.0], [2.0, 7.0, 0.0], [3.0, 5.0, 1.0]], dtype=np.float32)
    beta, counts = xs.xsvs_contrast(torch.from_numpy(frames).cuda(), grid, np.eye(3) * 10.0, [1, 3], 1, 1.0)
    assert list(counts) == [2]
    b = beta.cpu().numpy()
    # K=1: [1,1] -> 0; [2,0] -> 1; [3,1] -> (5 - 4)/4 = 1/4 ; mean 5/12
    # K=3: sums [6,2]: m1 = 4, m2 = 20 -> (20 - 16)/16 = 1/4
    assert abs(b[0, 0] - 5.0 / 12.0) < 1e-14
    assert abs(b[1, 0] - 0.25) < 1e-14


def test_config0_end_to_end_fp32(xs):
    traj, grid = wl.config0()
    p = torch.from_numpy(traj.pos).cuda()
    fd = torch.from_numpy(traj.f).cuda()
    I = xs.intensity(p, fd, traj.box, grid, "fp32")
    taus = list(range(1, 10))
    Ks = list(range(1, 11))
    R = wl.rings_for_plane(grid)
    g, mean = xs.g2(I.reshape(I.shape[0], -1), taus)
    beta, counts = xs.xsvs_contrast(I, grid, traj.box, Ks, R)
    xs.Context.get().sync_status()
    Iref = oracle.intensity(traj.pos, traj.f, traj.box, grid.miller())
    gref, mref = oracle.g2(Iref, taus)
    rings = oracle.ring_index(traj.box, grid.miller(), 1.0, R)
    bref, _ = oracle.xsvs_contrast(Iref, Ks, rings, R)
    # e_g2: relative L2 over all q != 0 pixels and delays (the norm-wise
    # analogue of e_I); the largest absolute deviation on pixels whose mean is
    # at least 1 % of the plane mean is bounded by the FP32 intensity error
    # there (a pixel 100x dimmer than average carries ~1e-7 sqrt(N)/|S| ~ 1e-6)
    nz = np.any(grid.miller() != 0, axis=1)
    gg = g.cpu().numpy()
    e_g2 = np.linalg.norm(gg[:, nz] - gref[:, nz]) / np.linalg.norm(gref[:, nz])
    assert e_g2 <= 1e-6, e_g2
    mask = mref >= 1e-2 * mref.mean()
    assert np.max(np.abs(gg[:, mask] - gref[:, mask])) <= 2e-5
    ok = counts >= 8
    e_b = np.max(np.abs(beta.cpu().numpy()[:, ok] - bref[:, ok]) / np.abs(bref[:, ok]))
    assert e_b <= 1e-6, e_b


def test_xsvs_over_pixel_shards_matches_the_whole(xs):
    # two shards of one plane (emulated ranks on one GPU): partial sums added,
    # as an all-reduce would, then finalized on the host
    import oracle as _oracle
    T, grid, box = 300, wl.centered_plane(48), np.eye(3) * 30.0
    n_rings = wl.rings_for_plane(grid)
    m = grid.miller()
    rings = _oracle.ring_index(box, m, 1.0, n_rings)
    g = torch.Generator(device="cuda").manual_seed(11)
    I = torch.rand((T, m.shape[0]), generator=g, device="cuda") + 0.1
    Ks = [1, 2, 5, 10, 50, 300]
    whole, counts = xs.xsvs_contrast(I.view(T, 1, grid.ny, grid.nx), grid, box, Ks, n_rings)
    sums, cnt = None, None
    for shard in (np.arange(m.shape[0]) % 3 == 0, np.arange(m.shape[0]) % 3 != 0):
        idx = torch.from_numpy(np.flatnonzero(shard)).cuda()
        s, c = xs.xsvs_partial(I[:, idx].contiguous(), rings[shard], n_rings, Ks)
        sums = s if sums is None else sums + s
        cnt = c if cnt is None else cnt + c
    xs.Context.get().sync_status()
    beta = xs.xsvs_finalize(sums, cnt, T, Ks)
    assert np.array_equal(cnt, counts)
    assert np.allclose(beta, whole.cpu().numpy(), rtol=1e-12, atol=0, equal_nan=True)
    ref, _ = _oracle.xsvs_contrast(I.cpu().numpy(), Ks, rings, n_rings)
    assert np.allclose(beta, ref, rtol=1e-9, atol=1e-12, equal_nan=True)
