"""The checked build (XS_BUILD_VARIANT=check, compiled with -DXS_BOUNDS_CHECK):
its kernels test their shared-memory, tensor-memory, workspace, record and
output indexes, and a failed test sets a bit of the device error word and
skips the access (no assert, no trap).

Run in child processes, since the variant is chosen when the package is
imported:
  * parity: the single path on both tile kinds (with a unit split along the
    atoms, so the partial-amplitude checks run), the batched path and the
    adjoint against the FP64 oracle (Sec. 3.1 direct method; the adjoint of
    Eq. 1), every call followed by a clean error word;
  * self-test: with XS_CHECK_SHORT_OUTPUT=1 the check admits one frame of I
    less than the buffers hold.  The last frame's writes fail the check and
    are skipped while every access stays inside the real buffers; the call
    reports XS_ERR_BOUNDS (7) and the frames before it are still right.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _case(seed, N, T, L, sigma=0.3):
    rng = np.random.default_rng(seed)
    base = rng.random((N, 3)) * L
    steps = rng.standard_normal((T, N, 3)) * sigma
    steps[0] = 0
    pos = (base[None] + np.cumsum(steps, axis=0)).astype(np.float32)
    f = np.where(rng.random(N) < 0.5, 1.0, 0.6).astype(np.float32)
    return pos, f, np.eye(3) * L


def _worker_parity(out):
    import torch
    import oracle
    from gpu_util import check_I
    from paper_2204_13241_gb300 import _native as nat, api as xs, workloads as wl

    out["lib"] = nat.library_path()
    ctx = xs.Context.get()
    res = []
    # (atoms, frames, grid, precision): a centred 128 x 128 tile; a ragged
    # 128 x 64 kind; 16,384 atoms on one tile, split along the atoms
    cases = [(4000, 3, wl.centered_plane(128), "fp16"),
             (3000, 3, wl.QGrid(-10, 150, -30, 50, 0, 1), "bf16"),
             (16384, 1, wl.QGrid(-64, 128, -64, 128, 0, 1), "fp16"),
             (2000, 2, wl.QGrid(-20, 40, -9, 64, -2, 3), "bf16")]
    for N, T, grid, prec in cases:
        pos, f, box = _case(N + T, N, T, 30.0)
        I, A = xs.intensity(torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda(), box, grid, prec,
                            want_amp=True)
        ctx.sync_status()
        m = grid.miller()
        S = oracle.amplitude(pos, f, box, m)
        e, e0, ep = check_I(I.reshape(T, -1).cpu().numpy(), np.abs(S) ** 2, m, prec, what="checked")
        res.append(["single", N, T, prec, e, ep])
    # batched: two trajectories on grids of both tile kinds
    trajs, grids, refs = [], [], []
    for seed, N, T, grid in [(1, 2500, 3, wl.centered_plane(128)), (2, 1800, 2, wl.QGrid(-64, 128, -20, 40, 0, 1))]:
        pos, f, box = _case(seed, N, T, 25.0)
        trajs.append((torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda(), box))
        grids.append(grid)
        refs.append((np.abs(oracle.amplitude(pos, f, box, grid.miller())) ** 2, grid.miller(), T))
    outs = xs.intensity_batched(trajs, grids, "fp16")
    ctx.sync_status()
    for o, (ref, m, T) in zip(outs, refs):
        e, e0, ep = check_I(o.reshape(T, -1).cpu().numpy(), ref, m, "fp16", what="checked batched")
        res.append(["batched", 0, T, "fp16", e, ep])
    # adjoint
    rng = np.random.default_rng(7)
    N, L = 1000, 18.0
    grid = wl.QGrid(-20, 40, -9, 300, 0, 1)
    pos = (rng.random((N, 3)) * L).astype(np.float32)
    f = rng.uniform(0.5, 1.5, N).astype(np.float32)
    G = rng.standard_normal(grid.n_pixels).astype(np.float32)
    amp = oracle.amplitude(pos, f, np.eye(3) * L, grid.miller())[0]
    Aa = np.stack([amp.real, amp.imag], axis=-1).astype(np.float32)
    g = xs.intensity_backward(torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda(), np.eye(3) * L, grid,
                              torch.from_numpy(Aa).cuda(), torch.from_numpy(G).cuda())
    ctx.sync_status()
    ref = oracle.grad_analytic(pos, f, np.eye(3) * L, grid.miller(), G.astype(np.float64),
                               amp=Aa[..., 0].astype(np.float64) + 1j * Aa[..., 1].astype(np.float64))
    err = float(np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref))
    assert err <= 1e-4, err
    res.append(["adjoint", N, 1, "split", err, err])
    out["cases"] = res


def _worker_short(out):
    import torch
    import oracle
    from paper_2204_13241_gb300 import _native as nat, api as xs, workloads as wl

    out["lib"] = nat.library_path()
    ctx = xs.Context.get()
    N, T = 3000, 3
    grid = wl.centered_plane(128)
    pos, f, box = _case(4, N, T, 30.0)
    I = torch.full((T, 1, grid.ny, grid.nx), -1.0, device="cuda")
    xs.intensity(torch.from_numpy(pos).cuda(), torch.from_numpy(f).cuda(), box, grid, "fp16", out=I)
    try:
        ctx.sync_status()
        out["status"] = 0
    except nat.XsError as ex:
        out["status"] = ex.status
        out["message"] = str(ex)
    Ih = I.reshape(T, -1).cpu().numpy()
    m = grid.miller()
    ref = np.abs(oracle.amplitude(pos[:T - 1], f, box, m)) ** 2
    nz = np.any(m != 0, axis=1)
    out["e_kept"] = max(float(np.linalg.norm(Ih[t, nz] - ref[t, nz]) / np.linalg.norm(ref[t, nz]))
                        for t in range(T - 1))
    out["last_untouched"] = bool(np.all(Ih[T - 1] == -1.0))
    # the error word was cleared and the context stays usable: a call on the
    # FP32 path, whose bounds the self-test leaves alone, is clean
    xs.intensity(torch.from_numpy(pos[:1].copy()).cuda(), torch.from_numpy(f).cuda(), box, grid, "fp32")
    try:
        ctx.sync_status()
        out["after"] = 0
    except nat.XsError as ex:
        out["after"] = ex.status


def _run(mode, short=False, timeout=900):
    env = dict(os.environ)
    env["XS_BUILD_VARIANT"] = "check"
    env.pop("XS_CHECK_SHORT_OUTPUT", None)
    if short:
        env["XS_CHECK_SHORT_OUTPUT"] = "1"
    env["PYTHONPATH"] = os.pathsep.join([ROOT, HERE] + [p for p in [env.get("PYTHONPATH")] if p])
    p = subprocess.run([sys.executable, os.path.abspath(__file__), mode], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=timeout)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def checked_lib():
    env = dict(os.environ, XS_BUILD_VARIANT="check")
    p = subprocess.run([sys.executable, "-c", "from paper_2204_13241_gb300 import build; build.build()"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stderr[-3000:]


def test_checked_build_matches_the_oracle_with_a_clean_error_word(checked_lib):
    r = _run("parity")
    assert "_build_check" in r["lib"]
    kinds = [c[0] for c in r["cases"]]
    assert kinds.count("single") == 4 and kinds.count("batched") == 2 and kinds.count("adjoint") == 1


def test_checked_build_reports_a_failed_check_and_skips_the_access(checked_lib):
    r = _run("short", short=True)
    assert "_build_check" in r["lib"]
    assert r["status"] == 7, r
    assert "bounds" in r["message"]
    assert r["last_untouched"], r
    assert r["e_kept"] <= 1e-4, r
    assert r["after"] == 0, r


if __name__ == "__main__":
    res = {}
    {"parity": _worker_parity, "short": _worker_short}[sys.argv[1]](res)
    print("RESULT " + json.dumps(res))
