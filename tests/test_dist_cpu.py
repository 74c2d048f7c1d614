"""Multi-rank paths on the CPU with two gloo ranks on 127.0.0.1:
  * the benchmark: the ranks agree on the slowest rank's time, and the
    whole-job value counts every rank's replica (weak scaling); the reference
    arm does no work on ranks other than 0;
  * XSVS over pixel shards: each rank's window sums per ring, all-reduced, go
    through the library's xs_xsvs_finalize and give the contrast of all pixels
    (the exchange of the sharded design, Sec. 2.3 Eq. bq_Iq)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        ms = 10.0 + 5.0 * rank                   # rank 1 is the slower one
        ms_max = bench.reduce_max(dist, ms, "cpu")
        q.put((r, w, ms_max, bench.job_value(1e9, w, ms_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms_max, value in out:
        assert w == 2 and ms_max == 15.0
        assert value == pytest.approx(1e9 * 2 / 15e-3)
    assert sorted(o[0] for o in out) == [0, 1]


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    # rank 0 of one: the oracle on a bounded sample, in the bench line's format
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == d["unit"] == "atom*pixel*frames/s"
    assert d["config"]["workload"] == "fcc256k_T1000_plane128"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def _shard_sums(I, ring, n_rings, Ks):
    # window sums per ring of one shard's pixels, laid out as xs_xsvs_partial writes them
    T = I.shape[0]
    rows = []
    for K in Ks:
        for w in range(T // K):
            x = I[w * K:(w + 1) * K].sum(axis=0)
            rows.append([[x[ring == r].sum(), (x[ring == r] ** 2).sum()] for r in range(1, n_rings + 1)])
    counts = np.array([(ring == r).sum() for r in range(1, n_rings + 1)], dtype=np.int64)
    return np.array(rows, dtype=np.float64), counts


def _xsvs_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2204_13241_gb300 import api as xs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)                       # every rank draws the same series
        T, P, n_rings, Ks = 40, 300, 6, [1, 3, 8, 40]
        I = rng.exponential(size=(T, P))
        ring = rng.integers(0, n_rings + 1, P).astype(np.int32)
        mine = np.arange(P) % world == rank                   # pixel shard of this rank
        sums, counts = _shard_sums(I[:, mine], ring[mine], n_rings, Ks)
        ts, tc = torch.from_numpy(sums), torch.from_numpy(counts)
        dist.all_reduce(ts)
        dist.all_reduce(tc)
        beta = xs.xsvs_finalize(ts.numpy(), tc.numpy(), T, Ks)
        ref, cref = oracle.xsvs_contrast(I, Ks, ring, n_rings)
        ok = bool(np.array_equal(tc.numpy(), cref) and np.allclose(beta, ref, rtol=1e-12, atol=0, equal_nan=True))
        q.put((rank, ok))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_pixels_for_xsvs_and_finalize_in_the_library():
    from paper_2204_13241_gb300 import build as xbuild
    xbuild.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_xsvs_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok in out), out


def _bench_shard_rank_main(rank, world, port, q):
    # the orchestration of `bench.py --shard pixels` with the GPU work replaced
    # by host sums: slabs of n_y rows, the whole ring layout on every rank,
    # the window sums all-reduced and finalized by the library
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2204_13241_gb300 import api as xs
    from paper_2204_13241_gb300 import workloads as wl

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = wl.centered_plane(24)
        box = np.eye(3) * 30.0
        R = wl.rings_for_plane(grid)
        T, Ks = 30, [1, 2, 5, 10, 30]
        rng = np.random.default_rng(11)                   # every rank draws the same series
        I = rng.exponential(size=(T, grid.n_pixels))
        slab, off, cnt = bench.shard_grid(grid, rank, world)
        m_full, m_slab = grid.miller(), slab.miller()
        same_pixels = bool(np.array_equal(m_full[off:off + cnt], m_slab))
        ring_full = xs.ring_index(grid, box, 1.0, R)
        ring_r = ring_full[off:off + cnt]
        counts_full = np.bincount(ring_full, minlength=R + 1)[1:].astype(np.int64)
        sums, _ = _shard_sums(I[:, off:off + cnt], ring_r, R, Ks)
        ts = torch.from_numpy(sums)
        dist.all_reduce(ts)
        beta = xs.xsvs_finalize(ts.numpy(), counts_full, T, Ks)
        ref, cref = oracle.xsvs_contrast(I, Ks, oracle.ring_index(box, m_full, 1.0, R), R)
        ok = bool(same_pixels and np.array_equal(counts_full, cref)
                  and np.allclose(beta, ref, rtol=1e-12, atol=0, equal_nan=True))
        q.put((rank, ok, cnt))
    finally:
        dist.destroy_process_group()


def test_bench_pixel_shards_on_two_gloo_ranks():
    from paper_2204_13241_gb300 import build as xbuild
    xbuild.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_bench_shard_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in out), out
    assert sum(c for _, _, c in out) == 24 * 24


def test_shard_rows_cover_every_row_once():
    sys.path.insert(0, ROOT)
    import bench
    for n in (1, 7, 64, 128, 129):
        for world in (1, 2, 3, 8):
            parts = [bench.shard_rows(n, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == n
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
