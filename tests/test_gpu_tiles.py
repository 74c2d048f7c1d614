"""The two tile kinds of the tensor-core contraction and the autotuner that
picks between them (the direct method does not depend on how the q grid is
tiled: Sec. 3.1, Algorithm 1).  Every shape is checked against the FP64
oracle with both kinds forced through the tuner's cache, the tuner's choice
is kept per shape bucket and used by single and batched calls, and batched
calls with trajectories of both kinds match single calls."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_I, e_I, e_pix
from paper_2204_13241_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xs():
    from paper_2204_13241_gb300 import build
    build.build()
    from paper_2204_13241_gb300 import api
    return api


def _case(seed, N, T, L, sigma=0.3):
    rng = np.random.default_rng(seed)
    base = rng.random((N, 3)) * L
    steps = rng.standard_normal((T, N, 3)) * sigma
    steps[0] = 0
    pos = (base[None] + np.cumsum(steps, axis=0)).astype(np.float32)
    f = np.where(rng.random(N) < 0.5, 1.0, 0.6).astype(np.float32)
    return pos, f, np.eye(3) * L


SHAPES = [
    wl.centered_plane(64),                    # one 128 x 64 tile
    wl.QGrid(-10, 150, -30, 50, 0, 1),        # two x tiles, ragged y (not symmetric)
    wl.QGrid(-20, 40, -9, 64, -2, 3),         # a small volume
    wl.QGrid(0, 128, 5, 60, 1, 1),            # q_z != 0, ragged
]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("grid", SHAPES)
def test_small_tile_kind_against_oracle(xs, grid, prec):
    # grids with n_y <= 64 take the 128 x 64 tile by default
    assert xs.tuned_choice(3000, grid, prec)[0] == 1
    pos, f, box = _case(11 + grid.nx, 3000, 3, 27.0)
    p, fd = torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda()
    I, A = xs.intensity(p, fd, box, grid, prec, want_amp=True)
    xs.Context.get().sync_status()
    m = grid.miller()
    S = oracle.amplitude(pos, f, box, m)
    check_I(I.reshape(3, -1).cpu().numpy(), np.abs(S) ** 2, m, prec)


def test_kinds_agree_and_the_tuner_keeps_its_choice(xs):
    # a shape where both kinds apply: 40,000 atoms on a 128 x 64 plane
    pos, f, box = _case(5, 40000, 70, 60.0)
    grid = wl.QGrid(-64, 128, -32, 64, 0, 1)
    p, fd = torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda()
    I1 = xs.intensity(p, fd, box, grid, "fp16")   # default: kind 1
    xs.Context.get().sync_status()
    xs.tune(p, fd, box, grid, "fp16")
    kind, chunk = xs.tuned_choice(40000, grid, "fp16")
    assert kind in (0, 1) and chunk in (16, 32, 64)
    # the choice is kept per bucket: 33,000 atoms fall in the same power of two
    assert xs.tuned_choice(33000, grid, "fp16") == (kind, chunk)
    I2 = xs.intensity(p, fd, box, grid, "fp16")   # the tuned choice
    xs.Context.get().sync_status()
    m = grid.miller()
    ref = oracle.intensity(pos[[0, 69]], f, box, m)
    check_I(I1.reshape(70, -1).cpu().numpy()[[0, 69]], ref, m, "fp16")
    check_I(I2.reshape(70, -1).cpu().numpy()[[0, 69]], ref, m, "fp16")
    a, b = I1.reshape(70, -1).cpu().numpy(), I2.reshape(70, -1).cpu().numpy().astype(np.float64)
    assert e_I(a, b, m)[0] <= 1e-4 and e_pix(a, b, m) <= 2e-3


def test_batched_with_both_kinds_matches_single_calls(xs):
    cases = [(2500, 3, wl.centered_plane(64), 24.0), (4000, 2, wl.centered_plane(128), 30.0),
             (1800, 4, wl.QGrid(-10, 100, -20, 40, 1, 1), 20.0), (6000, 2, wl.centered_plane(192), 40.0)]
    trajs, grids, host = [], [], []
    for i, (N, T, grid, L) in enumerate(cases):
        pos, f, box = _case(60 + i, N, T, L)
        trajs.append((torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda(), box))
        grids.append(grid)
        host.append((pos, f, box))
    kinds = [xs.tuned_choice(t[0].shape[1], g, "bf16")[0] for t, g in zip(trajs, grids)]
    assert 0 in kinds and 1 in kinds
    outs = xs.intensity_batched(trajs, grids, "bf16")
    xs.Context.get().sync_status()
    for (p, fd, box), grid, I_b, (pos, f, _) in zip(trajs, grids, outs, host):
        I_s = xs.intensity(p, fd, box, grid, "bf16")
        xs.Context.get().sync_status()
        m = grid.miller()
        T = I_s.shape[0]
        ref_s = I_s.reshape(T, -1).cpu().numpy().astype(np.float64)
        got = I_b.reshape(T, -1).cpu().numpy()
        assert e_I(got, ref_s, m)[0] <= 1e-4 and e_pix(got, ref_s, m) <= 2e-3
        ref = oracle.intensity(pos[T - 1:T], f, box, m)
        check_I(got[T - 1:T], ref, m, "bf16", what=str(grid))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("N,T,grid", [
    (3000, 3, wl.QGrid(-30, 60, -70, 140, 0, 1)),     # 60 n_x: narrow 128 x 128 tiles, two y tiles
    (3000, 2, wl.QGrid(-100, 180, -40, 100, 0, 1)),   # the second x tile holds 52 rows
    (16384, 1, wl.QGrid(-25, 50, -64, 128, 0, 1)),    # one narrow unit split along the atoms
    (2000, 2, wl.QGrid(-12, 33, -20, 40, 1, 2)),      # 128 x 64 kind, 33 rows, q_z != 0
])
def test_narrow_tiles_against_oracle(xs, N, T, grid, prec):
    # tiles with at most 64 valid n_x rows build only those rows, 32 per CTA
    pos, f, box = _case(N + grid.nx, N, T, 26.0)
    p, fd = torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda()
    I, A = xs.intensity(p, fd, box, grid, prec, want_amp=True)
    xs.Context.get().sync_status()
    m = grid.miller()
    S = oracle.amplitude(pos, f, box, m)
    check_I(I.reshape(T, -1).cpu().numpy(), np.abs(S) ** 2, m, prec)
