#!/usr/bin/env python3
"""Throughput of the direct-method XPCS/XSVS hot path on GB300.

One step = the whole path over one batch: the intensity I(q,t) of every
frame on the detector plane (split-FP16 tensor-core contraction over atoms,
Sec. 3.1 Algorithm 1), its g2 on 64 log-spaced delays (Sec. 2.3) and its
XSVS contrast on 1-2-5 window lengths over unit |q| rings (Sec. 2.3).
Workload: 256,000-atom FCC crystal (a = 4 A, L = 160 A, thermal 0.15 A,
f in {1.0, 0.6}), 1,000 Brownian frames (0.05 A), 128 x 128 plane at n_z = 0.

Metric: atom*pixel*frames per second (N * P * T / step time), whole job.
With --gpus N (torchrun), every rank runs its own replica of the workload
(independent problems, no collective on the data path): weak scaling.

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "atom*pixel*frames/s"
FALLBACK_PEAK = {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}
# FP32 SIMT rate from the unit counts and the maximum SM clock (152 SMs x 128
# FP32 lanes x 2 flops x 2.07 GHz); nominal, the measured peaks carry none
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# issue rate in thread-instructions per second (152 SMs x 4 schedulers x 32
# lanes x 2.07 GHz), the bound of the FP32 direct kernel, which ncu puts at
# about 53 thread-instructions per atom*pixel*frame
ISSUE_PEAK_TINST = 152 * 4 * 32 * 2.07e9
DIRECT_INST_PER_UNIT = 53.0

# DRAM bytes (read + write) of one tc_kernel launch, from an ncu capture of
# the 160-frame case of the same workload (dram__bytes_read.sum +
# dram__bytes_write.sum: 656.34 MB + 14.66 MB), scaled by frames: the
# records read and the intensities written are per frame, the split pieces'
# partials (a few MB) are not.  Reported only while k_tc.cu is unchanged.
TC_TRAFFIC = {"k_tc_sha256_prefix": "245a3523b1588130", "bytes": 656344576 + 14661632, "frames": 160}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=1000, help="frames of the workload (default: all 1,000)")
    ap.add_argument("--precision", choices=["fp16", "bf16"], default="fp16")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-table1", action="store_true")
    ap.add_argument("--no-next", action="store_true", help="skip the ISF, Ewald-slice and species timings")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing on its own workload")
    ap.add_argument("--shard", choices=["replicas", "pixels"], default="replicas",
                    help="with several GPUs: every rank runs its own replica (default, weak scaling), or the "
                         "ranks split the detector's n_y rows (strong scaling: I and g2 local, XSVS window sums "
                         "all-reduced)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 4,000-atom FP32 and the 3.2-million-atom crystal entries")
    return ap.parse_args()


def _tc_traffic(frames: int):
    import hashlib
    src = os.path.join(ROOT, "paper_2204_13241_gb300", "csrc", "k_tc.cu")
    try:
        with open(src, "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    if not sha.startswith(TC_TRAFFIC["k_tc_sha256_prefix"]):
        return None
    return TC_TRAFFIC["bytes"] * frames / TC_TRAFFIC["frames"]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAK), "fallback"


class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock, power and throttle
    reasons.  The sampler starts shortly before the timed region, so its first
    samples can see an idle GPU: given the region's start and end (host wall
    clock), the summary keeps the samples stamped inside it, and it leaves out
    samples whose gpu_idle reason is active (all are kept if none is left)."""

    FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap",
              "clocks_event_reasons.gpu_idle"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.fh = None

    def start(self):
        self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", self.gpu_id], stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, t0: float | None = None, t1: float | None = None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.flush()
        self.fh.seek(0)
        rows = [ln.strip().split(",") for ln in self.fh.read().splitlines() if ln.strip()]
        os.unlink(self.fh.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        parsed = []
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm_v, mx_v = float(r[1]), float(r[2])
            except ValueError:
                continue
            try:
                pw = float(r[3])
            except ValueError:
                pw = float("nan")
            try:
                stamp = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                stamp = None
            active = {name for name, v in zip(names, r[5:9]) if v.lower().startswith("active")}
            idle = len(r) > 9 and r[9].lower().startswith("active")
            parsed.append((sm_v, mx_v, pw, active, idle, stamp))
        if not parsed:
            return None
        powers = [p[2] for p in parsed if p[2] == p[2]]
        inside = parsed
        if t0 is not None and t1 is not None:
            inside = [p for p in parsed if p[5] is not None and t0 <= p[5] <= t1] or parsed
        loaded = [p for p in inside if not p[4]] or inside
        reasons = set().union(*(p[3] for p in loaded))
        return {"sm_mhz": statistics.median(p[0] for p in loaded), "sm_max_mhz": max(p[1] for p in parsed),
                "reasons": sorted(reasons), "samples": len(loaded), "samples_total": len(parsed),
                "power_w_median": statistics.median(p[2] for p in loaded) if powers else None}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(dist, v: float, device) -> float:
    """Maximum of v over the ranks of the process group (v itself without one)."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: every rank runs its own replica of the workload
    (weak scaling), so the job processes world x units in the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def shard_rows(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous split of n rows over the ranks: (first row, rows) of `rank`;
    the first n % world ranks take one row more."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def shard_grid(grid, rank: int, world: int):
    """A rank's slab of a detector plane: its n_y rows, all n_x.  With x
    fastest in the pixel order, the slab is the contiguous pixel range
    [offset, offset + count) of the whole plane.  Returns (slab, offset,
    count)."""
    from paper_2204_13241_gb300.workloads import QGrid

    if grid.nz != 1:
        raise ValueError("pixel shards are slabs of a plane")
    s, c = shard_rows(grid.ny, rank, world)
    return QGrid(grid.nx0, grid.nx, grid.ny0 + s, c, grid.nz0, 1), s * grid.nx, c * grid.nx


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2204_13241_gb300 import workloads as wl

    oracle.build()
    traj, grid = wl.config1(keep=[0])
    m = grid.miller()
    n_pix = 1024
    rng = np.random.default_rng(7)
    cores = oracle.max_threads()
    per_step = traj.n_atoms * n_pix
    for _ in range(args.warmup):
        sel = rng.choice(m.shape[0], n_pix, replace=False)
        oracle.intensity(traj.pos[:1], traj.f, traj.box, m[sel])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sel = rng.choice(m.shape[0], n_pix, replace=False)
        oracle.intensity(traj.pos[:1], traj.f, traj.box, m[sel])
    dt = (time.perf_counter() - t0) / args.steps
    value = per_step / dt
    sample = f"frame 0, {n_pix} random pixels of the 128^2 plane, {traj.n_atoms} atoms, per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fcc256k_T1000_plane128", "n_atoms": traj.n_atoms, "n_frames": 1000,
                   "grid": "128x128 (n_z=0)", "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _roof_tensor(units, ms, peaks, what):
    peak = float(peaks[0].get("bf16_tflops_sustained", FALLBACK_PEAK["bf16_tflops_sustained"]))
    a = 8.0 * units / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
            "kernel": what, "kernel_ms_per_call": ms, "peak_source": f"{peaks[1]} bf16 sustained",
            "note": "8 algorithmic flops per atom*pixel*frame (one complex multiply-add)"}


def config_entries(xs, ctx, stream, peaks):
    """Entries for the 4,000-atom workload on the FP32 path (its whole step)
    and the 3.2-million-atom crystal; returns (entries, what the oracle checks
    later in the CPU-baseline leg)."""
    import torch
    from paper_2204_13241_gb300 import workloads as wl

    out, keep = {}, {}

    def ev_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        ctx.sync_status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        return e0.elapsed_time(e1) / reps, r

    def stage_ms(tag, fn, reps):
        """device time of the `tag` launches per call (library events)"""
        fn()
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read("")
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        ms, n = ctx.profile_read(tag)
        ctx.profile(False)
        return ms / reps

    # 4,000 atoms, 10 frames, 64^2 plane: intensity (FP32 direct), g2 on
    # delays 1..9, XSVS on K = 1..10 over unit rings
    tr0, g0 = wl.config0()
    p0 = torch.from_numpy(tr0.pos).cuda()
    f0 = torch.from_numpy(tr0.f).cuda()
    T0, P0 = tr0.pos.shape[0], g0.n_pixels
    R0 = wl.rings_for_plane(g0)
    taus0, Ks0 = list(range(1, 10)), list(range(1, 11))
    I0 = torch.empty((T0, 1, g0.ny, g0.nx), dtype=torch.float32, device="cuda")

    def step0():
        xs.intensity(p0, f0, tr0.box, g0, "fp32", out=I0)
        g, _ = xs.g2(I0.view(T0, -1), taus0)
        b, _ = xs.xsvs_contrast(I0, g0, tr0.box, Ks0, R0)
        return g, b

    ms0, (g0_out, b0_out) = ev_ms(step0, 20)
    d_ms = stage_ms("direct", lambda: xs.intensity(p0, f0, tr0.box, g0, "fp32", out=I0), 20)
    units0 = float(tr0.n_atoms) * P0 * T0
    ach = units0 * DIRECT_INST_PER_UNIT / (d_ms * 1e-3)
    out["c0_fp32_4000_atoms"] = {
        "workload": "4,000 atoms U[0,40)^3, f = 1, 10 Brownian frames (0.1 A), 64^2 plane; FP32 direct path; "
                    "step = intensity + g2 (tau 1..9) + XSVS (K 1..10)",
        "value": units0 / (ms0 * 1e-3), "unit": METRIC, "ms_per_step": ms0, "dtype": "f32",
        "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": ISSUE_PEAK_TINST / 1e12,
                     "unit": "T thread-instructions/s", "frac": ach / ISSUE_PEAK_TINST, "kernel": "direct_kernel",
                     "kernel_ms_per_call": d_ms,
                     "note": "about 53 thread-instructions per atom*pixel*frame (ncu); peak = 152 SMs x 4 "
                             "schedulers x 32 lanes x 2.07 GHz"}}
    keep["c0"] = (I0.view(T0, -1).cpu().numpy(), g0_out.cpu().numpy(), b0_out.cpu().numpy(), taus0, Ks0, R0, tr0, g0)
    del p0, f0

    # 3.2-million-atom crystal: 32 frames of the 512^2 plane streamed from
    # pinned host memory (host in, device out), the 128^3 volume on one frame
    nf4 = 32
    tr4, g4 = wl.config4(keep=range(nf4))
    N4 = tr4.n_atoms
    pos_h = torch.from_numpy(tr4.pos).pin_memory()
    f_h = torch.from_numpy(tr4.f).pin_memory()
    I4 = torch.empty((nf4, 1, g4.ny, g4.nx), dtype=torch.float32, device="cuda")
    ms4, _ = ev_ms(lambda: xs.intensity(pos_h, f_h, tr4.box, g4, "fp16", out=I4), 2)
    units4 = float(N4) * g4.n_pixels * nf4
    tc4 = stage_ms("tc", lambda: xs.intensity(pos_h, f_h, tr4.box, g4, "fp16", out=I4), 2)
    vol = wl.centered_volume(128)
    p1 = torch.from_numpy(tr4.pos[:1]).cuda()
    f1 = f_h.cuda()
    Iv = torch.empty((1, vol.nz, vol.ny, vol.nx), dtype=torch.float32, device="cuda")
    msv, _ = ev_ms(lambda: xs.intensity(p1, f1, tr4.box, vol, "fp16", out=Iv), 3)
    tcv = stage_ms("tc", lambda: xs.intensity(p1, f1, tr4.box, vol, "fp16", out=Iv), 3)
    unitsv = float(N4) * vol.n_pixels
    # g2 and XSVS at the workload's correlation size: 10,000 frames of the
    # 512^2 plane (a seeded speckle series with the ring's AR(1) correlation)
    T4 = 10_000
    n_rings4 = wl.rings_for_plane(g4)
    ring_h = xs.ring_index(g4, tr4.box, 1.0, n_rings4)
    rho = torch.from_numpy((0.3 + 0.65 * ring_h / n_rings4).astype(np.float32))
    Is = wl.speckle_series(wl.SEED_BASE + 40, T4, rho, "cuda")
    taus4 = [int(t) for t in wl.log_delays(T4)]
    Ks4 = [int(k) for k in wl.window_list_125(1000)]
    ms_g2, (g4_out, _) = ev_ms(lambda: xs.g2(Is, taus4), 2)
    ms_xs, (b4_out, _) = ev_ms(lambda: xs.xsvs_contrast(Is.view(T4, 1, g4.ny, g4.nx), g4, tr4.box, Ks4, n_rings4), 2)
    out["c4_crystal_3_2M_atoms"] = {
        "workload": "FCC a = 4 A, L = 400 A, 20% vacancies (3,200,000 atoms), thermal 0.2 A, Brownian frames "
                    "(0.02 A); split FP16",
        "plane_512_streamed": {"frames": nf4, "value": units4 / (ms4 * 1e-3), "unit": METRIC, "ms_per_call": ms4,
                               "h2d_bytes_per_call": int(tr4.pos.nbytes + tr4.f.nbytes),
                               "roofline": _roof_tensor(units4, tc4, peaks, "tc_kernel (all launches of one call: "
                                                        "the frames are streamed in chunks of growing size)")},
        "volume_128^3": {"frames": 1, "value": unitsv / (msv * 1e-3), "unit": METRIC, "ms_per_call": msv,
                         "roofline": _roof_tensor(unitsv, tcv, peaks, "tc_kernel")},
        "correlations_10000_frames_512^2": {"g2_ms": ms_g2, "n_tau": len(taus4), "xsvs_ms": ms_xs,
                                            "window_lengths": Ks4, "rings": n_rings4,
                                            "input": "seeded AR(1) speckle series with the workload's shape "
                                                     "(10,000 x 512^2; the 10,000 crystal frames would be 384 GB "
                                                     "of positions)"}}
    rng = np.random.default_rng(4)
    m4 = g4.miller()
    pix4 = np.unique(np.concatenate([np.flatnonzero(np.all(m4 == 0, axis=1)), rng.choice(m4.shape[0], 96, replace=False)]))
    mv = vol.miller()
    pixv = np.unique(np.concatenate([np.flatnonzero(np.all(mv == 0, axis=1)), rng.choice(mv.shape[0], 96, replace=False)]))
    pix_c = rng.choice(m4.shape[0], 256, replace=False)
    keep["c4"] = dict(tr=tr4, g=g4, vol=vol, pix=pix4, pixv=pixv,
                      I=I4.view(nf4, -1)[[0, nf4 - 1]][:, torch.from_numpy(pix4).cuda()].cpu().numpy(),
                      Iv=Iv.view(1, -1)[:, torch.from_numpy(pixv).cuda()].cpu().numpy(),
                      Is=Is[:, torch.from_numpy(pix_c).cuda()].cpu().numpy(), pix_c=pix_c,
                      g2=g4_out[:, torch.from_numpy(pix_c).cuda()].cpu().numpy(), taus=taus4)
    cnt_r = np.bincount(ring_h, minlength=n_rings4 + 1)
    sel_r = [r for r in (1, 50, 181, 300, n_rings4) if cnt_r[r] >= 8]
    sel = np.flatnonzero(np.isin(ring_h, sel_r))
    keep["c4"].update(Ir=Is[:, torch.from_numpy(sel).cuda()].cpu().numpy(), ring_sel=ring_h[sel], rings_pick=sel_r,
                      beta=b4_out.cpu().numpy(), Ks=Ks4, n_rings=n_rings4)
    del Is, I4, Iv, p1, f1, pos_h
    torch.cuda.empty_cache()
    return out, keep


def config_accuracy(entries, keep, ref0):
    """Errors of the entries of config_entries against the FP64 oracle (run in
    the CPU-baseline leg)."""
    import oracle

    I0, g0_out, b0_out, taus0, Ks0, R0, tr0, g0 = keep["c0"]
    m0 = g0.miller()
    nz0 = np.any(m0 != 0, axis=1)
    e_I0 = max(float(np.linalg.norm(I0[t, nz0] - ref0[t, nz0]) / np.linalg.norm(ref0[t, nz0])) for t in range(I0.shape[0]))
    e_pix0 = max(float(np.max(np.abs(I0[t, nz0] - ref0[t, nz0]) / np.maximum(ref0[t, nz0], ref0[t, nz0].mean())))
                 for t in range(I0.shape[0]))
    # end to end: the oracle's g2 and contrast of the oracle's intensity
    gref, _ = oracle.g2(ref0, taus0)
    e_g2_0 = float(np.linalg.norm(g0_out[:, nz0] - gref[:, nz0]) / np.linalg.norm(gref[:, nz0]))
    rings0 = oracle.ring_index(tr0.box, m0, 1.0, R0)
    bref, cref = oracle.xsvs_contrast(ref0, Ks0, rings0, R0)
    ok = cref >= 8
    e_b0 = float(np.max(np.abs(b0_out[:, ok] - bref[:, ok]) / np.abs(bref[:, ok])))
    entries["c0_fp32_4000_atoms"]["accuracy"] = {
        "e_I": e_I0, "e_pix": e_pix0, "e_g2": e_g2_0, "e_beta": e_b0, "target": 1e-6,
        "against": "FP64 oracle, every frame and pixel; g2 and beta end to end (oracle g2 and beta of the "
                   "oracle's intensity)"}
    k = keep["c4"]
    tr4 = k["tr"]
    ref = oracle.intensity(tr4.pos[[0, tr4.pos.shape[0] - 1]], tr4.f, tr4.box, k["g"].miller()[k["pix"]])
    refv = oracle.intensity(tr4.pos[:1], tr4.f, tr4.box, k["vol"].miller()[k["pixv"]])

    def errs(I, r, m):
        nz = np.any(m != 0, axis=1)
        e = max(float(np.linalg.norm(I[t, nz] - r[t, nz]) / np.linalg.norm(r[t, nz])) for t in range(r.shape[0]))
        ep = max(float(np.max(np.abs(I[t, nz] - r[t, nz]) / np.maximum(r[t, nz], r[t, nz].mean())))
                 for t in range(r.shape[0]))
        z = ~nz
        e0 = float(np.max(np.abs(I[:, z] - r[:, z]) / r[:, z])) if z.any() else 0.0
        return e, ep, e0

    e4, ep4, e04 = errs(k["I"].astype(np.float64), ref, k["g"].miller()[k["pix"]])
    ev, epv, e0v = errs(k["Iv"].astype(np.float64), refv, k["vol"].miller()[k["pixv"]])
    gr, _ = oracle.g2(k["Is"], k["taus"])
    e_g2 = float(np.max(np.abs(k["g2"] - gr) / np.abs(gr)))
    bo, co = oracle.xsvs_contrast(k["Ir"], k["Ks"], k["ring_sel"], k["n_rings"])
    cols = [r - 1 for r in k["rings_pick"]]
    e_b = float(np.max(np.abs(k["beta"][:, cols] - bo[:, cols]) / np.abs(bo[:, cols])))
    c4 = entries["c4_crystal_3_2M_atoms"]
    c4["plane_512_streamed"]["accuracy"] = {"e_I": e4, "e_pix": ep4, "e_q0": e04, "frames": [0, 31],
                                            "pixels": int(len(k["pix"]))}
    c4["volume_128^3"]["accuracy"] = {"e_I": ev, "e_pix": epv, "e_q0": e0v, "pixels": int(len(k["pixv"]))}
    c4["correlations_10000_frames_512^2"]["accuracy"] = {
        "e_g2_max_rel": e_g2, "g2_pixels": 256, "e_beta_max_rel": e_b, "beta_rings": k["rings_pick"],
        "against": "oracle g2 and beta of the same series (stage parity)"}


def run_ours(args):
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        # NCCL's initialisation log names the communicator's ranks
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return reduce_max(dist, v, "cuda")

    from paper_2204_13241_gb300 import build as xbuild
    from paper_2204_13241_gb300 import workloads as wl

    # rank 0 builds; the others wait for it instead of racing on the same files
    if rank == 0:
        xbuild.build()
    if dist is not None:
        dist.barrier()
    if not xbuild.up_to_date():
        raise RuntimeError("libxs.so is not built")
    from paper_2204_13241_gb300 import api as xs

    traj, grid = wl.config1(n_frames=args.frames)
    T, N, P = traj.pos.shape[0], traj.n_atoms, grid.n_pixels
    taus = [int(t) for t in wl.log_delays(T, 64)]
    Ks = [int(k) for k in wl.window_list_125(T)]
    R = wl.rings_for_plane(grid)
    box = traj.box
    pos_d = torch.from_numpy(traj.pos).to(f"cuda:{dev}")
    f_d = torch.from_numpy(traj.f).to(f"cuda:{dev}")
    ctx = xs.Context.get()
    sharded = args.shard == "pixels"
    if sharded:
        # this rank's n_y rows; every rank knows the whole ring layout, so
        # only the XSVS window sums are exchanged
        grid_r, p_off, p_cnt = shard_grid(grid, rank, world)
        ring_full = xs.ring_index(grid, box, 1.0, R)
        ring_r = ring_full[p_off:p_off + p_cnt]
        counts_full = np.bincount(ring_full, minlength=R + 1)[1:].astype(np.int64)
    else:
        grid_r, p_off, p_cnt = grid, 0, P
    I = torch.empty((T, 1, grid_r.ny, grid_r.nx), dtype=torch.float32, device="cuda")

    def step(pos, f):
        xs.intensity(pos, f, box, grid_r, args.precision, out=I)
        g, mean = xs.g2(I.view(T, -1), taus)
        if not sharded:
            beta, counts = xs.xsvs_contrast(I, grid, box, Ks, R)
            return g, mean, beta
        sums, _ = xs.xsvs_partial(I.view(T, -1), ring_r, R, Ks)
        if dist is not None:
            dist.all_reduce(sums)
        beta = xs.xsvs_finalize(sums, counts_full, T, Ks)
        return g, mean, beta

    for _ in range(max(args.warmup, 1)):
        step(pos_d, f_d)
    ctx.sync_status()

    # ---- timed region: inputs resident in HBM (7 GB of positions and phase
    # records per step, far above the 129 MB L2) -------------------------------
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else str(dev))
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    ctx.profile_read("")
    launches0 = ctx.launch_count()
    barrier()
    sampler.start()
    time.sleep(0.3)
    wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(pos_d, f_d)  # the last step's g2 and beta are checked against the oracle below
    ev1.record(stream)
    ev1.synchronize()
    wall1 = time.time()
    clocks = sampler.stop(wall0, wall1)
    barrier()
    I_step = I.clone()  # the timed step's intensity, for the accuracy check
    launches = ctx.launch_count() - launches0
    tc_ms, tc_n = ctx.profile_read("tc")
    # per-stage device time per step (library events around each stage's launches)
    breakdown = {"tc_kernel": tc_ms / args.steps}
    for tag in ("split_finish", "phase", "g2", "xsvs"):
        t_ms, _ = ctx.profile_read(tag)
        breakdown[tag] = t_ms / args.steps
    all_ms, all_n = ctx.profile_read("")
    breakdown["other"] = all_ms / args.steps
    all_ms += sum(v for k, v in breakdown.items() if k not in ("tc_kernel", "other")) * args.steps
    ctx.profile(False)
    ctx.sync_status()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms)
    units = float(N) * p_cnt * T          # this rank's atom*pixel*frames per step
    # replicas: every rank's units count; pixel shards: the ranks together do
    # the plane once per step
    value = job_value(units, world, ms) if not sharded else float(N) * P * T / (ms * 1e-3)

    peaks, peak_src = _peaks()
    tc_launch_ms = tc_ms / max(tc_n, 1)
    alg_flops = 8.0 * units           # one complex multiply-add per atom*pixel*frame
    exe_flops = 24.0 * units          # 4 real products x 3 split passes x 2 flops
    peak = float(peaks.get("bf16_tflops_sustained", FALLBACK_PEAK["bf16_tflops_sustained"]))
    achieved = alg_flops / (tc_launch_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": _tc_traffic(T),
                "traffic_note": "ncu DRAM bytes (read + write) of a 160-frame launch, scaled by frames; "
                                "algorithmic bytes per launch = T x (N x 16 B records + P x 4 B)",
                "algorithmic_bytes": float(T) * (N * 16.0 + P * 4.0),
                "kernel": "tc_kernel (split-FP16 contraction)", "kernel_ms_per_launch": tc_launch_ms,
                "peak_source": f"{peak_src} bf16 sustained (fp16 dense rate = bf16)",
                "executed_tflops": exe_flops / (tc_launch_ms * 1e-3) / 1e12,
                "executed_frac": exe_flops / (tc_launch_ms * 1e-3) / 1e12 / peak,
                "share_of_step": tc_ms / max(tc_ms + all_ms, 1e-9)}

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f16-split (hi+lo), f32 accumulate", "data": "synthetic",
            "config": {"workload": "fcc256k_T1000_plane128", "n_atoms": N, "n_frames": T,
                       "grid": f"{grid.nx}x{grid.ny} (n_z=0)", "precision": f"split_{args.precision}",
                       "n_tau": len(taus), "window_lengths": Ks, "rings": R,
                       "l2": "inputs larger than L2 (3.1 GB positions + 4.1 GB phase records read per step)",
                       "parallelism": (f"pixel shards x{world} (n_y rows, XSVS sums all-reduced)" if sharded
                                       else f"replicas x{world}")},
            "roofline": roofline, "gpu_launches": launches, "clocks": clocks,
            "stage_ms_per_step": {k: round(v, 4) for k, v in breakdown.items()}}

    # ---- pixel shards: the same plane on one GPU gives the same g2 and beta
    if sharded:
        g_sh, _, b_sh = res
        I_full = xs.intensity(pos_d, f_d, box, grid, args.precision)
        g_full, _ = xs.g2(I_full.view(T, -1), taus)
        b_full, _ = xs.xsvs_contrast(I_full, grid, box, Ks, R)
        ctx.sync_status()
        g_ref = g_full[:, p_off:p_off + p_cnt].cpu().numpy()
        b_ref = b_full.cpu().numpy()
        okr = counts_full >= 8
        d_g = float(np.max(np.abs(g_sh.cpu().numpy() - g_ref) / np.abs(g_ref)))
        d_b = float(np.max(np.abs(np.asarray(b_sh)[:, okr] - b_ref[:, okr]) / np.abs(b_ref[:, okr])))
        d_g, d_b = max_over_ranks(d_g), max_over_ranks(d_b)
        line["shard_check"] = {
            "g2_max_rel_vs_one_gpu": d_g, "beta_max_rel_vs_one_gpu": d_b,
            "note": "each rank's g2 of its rows and the all-reduced beta against the whole plane computed on "
                    "the rank's own GPU; a slab's tile layout differs from the plane's, so the FP32 "
                    "accumulation differs in the last bits"}
        del I_full

    # ---- end to end through the public API with host buffers ------------------
    if not args.no_e2e:
        pos_h = torch.from_numpy(traj.pos).pin_memory()
        f_h = torch.from_numpy(traj.f).pin_memory()
        I_h = torch.empty(I.shape, dtype=torch.float32).pin_memory()
        g_h = torch.empty((len(taus), p_cnt), dtype=torch.float64).pin_memory()
        b_h = torch.empty((len(Ks), R), dtype=torch.float64).pin_memory()

        side = torch.cuda.Stream()

        def e2e_step():
            if sharded:
                # pixel shards: this rank's rows streamed from host positions;
                # beta arrives on the host through the finalize
                g, _, beta = step(pos_h, f_h)
                I_h.copy_(I, non_blocking=True)
                g_h.copy_(g, non_blocking=True)
                b_h.copy_(torch.from_numpy(np.asarray(beta)))
                torch.cuda.current_stream().synchronize()
                return
            xs.intensity(pos_h, f_h, box, grid, args.precision, out=I)
            # the intensity goes back to the host on a side stream while g2
            # and the contrast run; the next step waits for it before it
            # writes I again
            done = torch.cuda.Event()
            done.record(stream)
            side.wait_event(done)
            with torch.cuda.stream(side):
                I_h.copy_(I, non_blocking=True)
            g, mean = xs.g2(I.view(T, -1), taus)
            beta, counts = xs.xsvs_contrast(I, grid, box, Ks, R)
            g_h.copy_(g, non_blocking=True)
            b_h.copy_(beta, non_blocking=True)
            stream.wait_stream(side)

        # the host link's copy rate on this machine (pinned, 256 MB, best of 3),
        # outside the timed region: the e2e figure is bound by it where it
        # is slow
        link = torch.empty(1 << 26, dtype=torch.float32).pin_memory()
        link_d = torch.empty(1 << 26, dtype=torch.float32, device=dev)
        link_gbs = 0.0
        for _ in range(3):
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            link_d.copy_(link, non_blocking=True)
            l1.record(stream)
            l1.synchronize()
            link_gbs = max(link_gbs, link.numel() * 4 / (l0.elapsed_time(l1) * 1e-3) / 1e9)
        del link, link_d
        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier()
        # each step timed on its own as well (synchronised at its end), so a
        # step stalled by the host shows in the spread beside the mean
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(args.steps):
            ts = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            step_ms.append((time.perf_counter() - ts) * 1e3)
        barrier()
        e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)
        ctx.sync_status()
        h2d = traj.pos.nbytes + traj.f.nbytes
        d2h = I_h.numel() * 4 + g_h.numel() * 8 + b_h.numel() * 8
        if sharded:
            d2h += sum(T // k for k in Ks) * R * 2 * 8   # the all-reduced window sums read by the finalize
        e_val = job_value(units, world, e_ms) if not sharded else float(N) * P * T / (e_ms * 1e-3)
        line["e2e"] = {"value": e_val, "unit": METRIC, "ms_per_step": e_ms,
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "host_to_device_gbs": link_gbs,
                       "step_ms_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)]}
        del pos_h

    # ---- plain FP32 direct-sum kernel on the same workload (first 32 frames) ---
    if not args.no_fp32 and rank == 0:
        nf = min(32, T)
        sub = pos_d[:nf].contiguous()
        I32 = torch.empty((nf, 1, grid.ny, grid.nx), dtype=torch.float32, device="cuda")
        xs.intensity(sub, f_d, box, grid, "fp32", out=I32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xs.intensity(sub, f_d, box, grid, "fp32", out=I32)
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        rate32 = float(N) * P * nf / (e0.elapsed_time(e1) * 1e-3)
        # the factorised FP32 kernel (same accuracy class) on the same frames
        xs.intensity(sub, f_d, box, grid, "fp32f", out=I32)
        torch.cuda.synchronize()
        e0.record(stream)
        xs.intensity(sub, f_d, box, grid, "fp32f", out=I32)
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        rate32f = float(N) * P * nf / (e0.elapsed_time(e1) * 1e-3)
        ours_rate = float(N) * P * T / (tc_launch_ms * 1e-3)
        line["fp32_direct"] = {"value": rate32, "unit": METRIC, "frames": nf,
                               "tc_kernel_rate": ours_rate, "speedup_tc_vs_fp32": ours_rate / rate32,
                               "fp32_factored": {"value": rate32f, "unit": METRIC,
                                                 "fma_tflops": 8.0 * rate32f / 1e12,
                                                 "of_fp32_peak": 8.0 * rate32f / 1e12 / FP32_PEAK_TFLOPS,
                                                 "note": "one complex multiply-add (4 FP32 FMAs) per unit; "
                                                         "nominal FP32 peak from unit counts and clocks"}}

    # ---- the paper's own timing setting (Table 1): 4,000 atoms in a
    # 59.19 A box, one q, an 81^2 slice and an 81^3 grid per frame, and the FFT
    # method on a 512^3 grid (the next power of two above the paper's 400)
    if not args.no_table1 and rank == 0:
        rng = np.random.default_rng(wl.SEED_BASE + 7)
        Lar, Nar, Tar = 59.19, 4000, 4
        pos_ar = torch.from_numpy((rng.random((Tar, Nar, 3)) * Lar).astype(np.float32)).cuda()
        f_ar = torch.ones(Nar, device="cuda")
        box_ar = np.eye(3) * Lar

        def per_frame(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            ctx.sync_status()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            ctx.sync_status()
            return e0.elapsed_time(e1) / reps / Tar * 1e-3

        g1 = wl.QGrid(5, 1, 3, 1, 0, 1)
        g81 = wl.QGrid(-40, 81, -40, 81, 0, 1)
        v81 = wl.QGrid(-40, 81, -40, 81, -40, 81)
        t_q = per_frame(lambda: xs.intensity(pos_ar, f_ar, box_ar, g1, "fp32"))
        t_s = per_frame(lambda: xs.intensity(pos_ar, f_ar, box_ar, g81, "fp16"))
        t_v = per_frame(lambda: xs.intensity(pos_ar, f_ar, box_ar, v81, "fp16"))
        t_f = per_frame(lambda: xs.intensity_fft(pos_ar, f_ar, box_ar, g81, 512, 2.0 * Lar / 512), reps=1)
        line["paper_table1"] = {
            "workload": "4,000 atoms uniform in a 59.19 A box (synthetic stand-in for the paper's Ar frame), f = 1",
            "seconds_per_frame": {"direct_single_q_fp32": t_q, "direct_81x81_slice_split_fp16": t_s,
                                  "direct_81x81x81_grid_split_fp16": t_v,
                                  "fft_method_512^3_fp64_eta_2_grid_steps": t_f},
            "paper_seconds_per_frame_32_cpus": {"direct_single_q": 0.0015, "direct_81x81_slice": 4.1836,
                                                "direct_81x81x81_grid": 416.8243, "fft_method_n400": 0.4527},
            "note": "paper: Table 1, 32 CPUs (model unstated), its own Ar frames; context, not a like-for-like ratio"}
        del pos_ar
        torch.cuda.empty_cache()

    # ---- the rows beyond the hot path, on the same crystal: per-species form
    # factors, the Ewald-sphere slice through the point path, and the
    # intermediate scattering function with its Siegert contrast
    def ms_per_call(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ctx.sync_status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        return e0.elapsed_time(e1) / reps

    keep_tables = {}
    if not args.no_next and rank == 0:
        nf = min(100, T)
        sub = pos_d[:nf].contiguous()
        t_plane = ms_per_call(lambda: xs.intensity(sub, f_d, box, grid, args.precision))
        plane_units = float(N) * P * nf
        # two species (alternate atoms) with synthetic four-Gaussian form factors
        species = np.arange(N, dtype=np.int32) % 2
        coef = np.array([[8.0, 12.0, 6.0, 1.5, 3.0, 40.0, 1.0, 90.0, 0.5],
                         [4.0, 20.0, 2.5, 4.0, 1.2, 0.6, 0.8, 60.0, 0.3]], dtype=np.float64)
        t_sp = ms_per_call(lambda: xs.intensity_species(sub, f_d, species, coef, box, grid, args.precision))
        # Ewald slice: beam along z, wavelength 1 A, over the 128 x 128 detector window
        k_in = [0.0, 0.0, 2.0 * math.pi / 1.0]
        mil, valid = xs.ewald_points(box, k_in, grid.nx0, grid.nx, grid.ny0, grid.ny)
        mil = mil[valid]
        t_pt = ms_per_call(lambda: xs.intensity_points(sub, f_d, box, mil, args.precision))
        # ISF on the amplitudes of the full series, same delays as g2
        _, amp = xs.intensity(pos_d, f_d, box, grid, args.precision, want_amp=True)
        sum_f2 = float((traj.f.astype(np.float64) ** 2).sum())
        t_isf = ms_per_call(lambda: xs.isf(amp, taus, sum_f2))
        Kmax = max(Ks)
        _, Fh = xs.isf(amp, list(range(Kmax)), sum_f2)
        t_cf = ms_per_call(lambda: xs.contrast_from_isf(Fh, grid, box, Ks, R))
        pairs = float(P) * sum(T - t for t in taus)
        # the FP64 table builder (every entry from sincospi of its exact turn
        # count) against the default seeds and rotations, same 100 frames
        ctx.set_table_builder(True)
        try:
            t_ex = ms_per_call(lambda: xs.intensity(sub, f_d, box, grid, args.precision))
            I_ex100 = xs.intensity(sub[:1].contiguous(), f_d, box, grid, args.precision).reshape(-1).cpu()
        finally:
            ctx.set_table_builder(False)
        I_rec100 = xs.intensity(sub[:1].contiguous(), f_d, box, grid, args.precision).reshape(-1).cpu()
        keep_tables.update(exact=I_ex100.numpy(), rec=I_rec100.numpy())
        line["next_rows"] = {
            "frames": nf,
            "table_builders": {"recurrence_ms_per_call": t_plane, "fp64_sincospi_ms_per_call": t_ex,
                               "slowdown": t_ex / t_plane,
                               "what": "default: FP32 seeds and rotations per run of n; option: FP64 sincospi "
                                       "of every entry's exact turn count"},
            "plane_reference": {"value": plane_units / (t_plane * 1e-3), "unit": METRIC, "ms_per_call": t_plane},
            "species_form_factors": {"value": plane_units / (t_sp * 1e-3), "unit": METRIC, "ms_per_call": t_sp,
                                     "species": 2, "coefficients": "synthetic four-Gaussian sums"},
            "ewald_slice_points": {"value": float(N) * mil.shape[0] * nf / (t_pt * 1e-3),
                                   "unit": "atom*point*frames/s", "ms_per_call": t_pt,
                                   "points": int(mil.shape[0]),
                                   "n_z_planes": int(np.unique(mil[:, 2]).size),
                                   "beam": "along z, wavelength 1 A, 128 x 128 detector window"},
            "isf": {"value": pairs / (t_isf * 1e-3), "unit": "pixel*delay*frame products/s",
                    "ms_per_call": t_isf, "frames": T, "n_tau": len(taus)},
            "contrast_from_isf": {"ms_per_call": t_cf, "delays": Kmax, "window_lengths": len(Ks)}}
        del sub, amp, Fh
        torch.cuda.empty_cache()

    # ---- the adjoint on its own workload: 100,000 atoms, a 256^2 plane, one
    # frame, L = sum_q w_q (I - I_target)^2 with w_q = 1 / (1 + |q|^2)
    if not args.no_adjoint and rank == 0:
        traj3, target3, grid3 = wl.config3()
        p3 = torch.from_numpy(traj3.pos[0]).cuda()
        f3 = torch.from_numpy(traj3.f).cuda()
        It = xs.intensity(torch.from_numpy(target3[0]).cuda(), f3, traj3.box, grid3, "fp32").reshape(-1)
        q2 = ((2.0 * math.pi / traj3.L) ** 2) * (grid3.miller().astype(np.float64) ** 2).sum(axis=1)
        w3 = torch.from_numpy((1.0 / (1.0 + q2)).astype(np.float32)).cuda()
        I3, A3 = xs.intensity(p3, f3, traj3.box, grid3, "fp32", want_amp=True)
        G3 = (2.0 * w3 * (I3.reshape(-1) - It)).contiguous()
        A3 = A3.reshape(-1, 2).contiguous()
        # calls of a fraction of a millisecond: 20 back to back, so that the
        # host's work for the first call is not a tenth of the figure
        t_b = ms_per_call(lambda: xs.intensity_backward(p3, f3, traj3.box, grid3, A3, G3), reps=20)
        t_f32 = ms_per_call(lambda: xs.intensity(p3, f3, traj3.box, grid3, "fp32", want_amp=True))
        t_f32f = ms_per_call(lambda: xs.intensity(p3, f3, traj3.box, grid3, "fp32f", want_amp=True), reps=20)
        t_f16 = ms_per_call(lambda: xs.intensity(p3, f3, traj3.box, grid3, args.precision, want_amp=True),
                            reps=20)
        units3 = float(traj3.n_atoms) * grid3.n_pixels
        peaks3, src3 = _peaks()
        peak3 = float(peaks3.get("bf16_tflops_sustained", FALLBACK_PEAK["bf16_tflops_sustained"]))
        achieved3 = 16.0 * units3 / (t_b * 1e-3) / 1e12   # two complex multiply-adds per atom*pixel
        line["adjoint"] = {
            "workload": "100,000 atoms U[0,120)^3, 256^2 plane, one frame",
            "backward_ms": t_b, "value": units3 / (t_b * 1e-3), "unit": "atom*pixel/s",
            "forward_fp32_with_amp_ms": t_f32, "forward_fp32_factored_with_amp_ms": t_f32f,
            f"forward_split_{args.precision}_with_amp_ms": t_f16,
            "fitting_step_ms": t_f32f + t_b,
            "roofline": {"bound": "tensor", "achieved": achieved3, "peak": peak3, "unit": "TFLOP/s",
                         "frac": achieved3 / peak3, "executed_frac": 3.0 * achieved3 / peak3,
                         "peak_source": f"{src3} bf16 sustained",
                         "note": "16 flops per atom*pixel (Z and Z_y, one complex multiply-add each), split BF16 "
                                 "in 3 passes; FP32 SIMT rate for comparison: "
                                 f"{FP32_PEAK_TFLOPS:.1f} TFLOP/s nominal"}}
        del p3, f3, It, I3, A3, G3
        torch.cuda.empty_cache()

    # ---- the batched workload: 64 ideal-gas trajectories in one persistent launch
    if not args.no_batched and rank == 0:
        del pos_d
        torch.cuda.empty_cache()
        params = wl.config2_params()
        trajs, grids = [], []
        for prm in params:
            trajs.append(wl.gas_on_device(prm, "cuda"))
            grids.append(wl.centered_plane(prm["side"]))
        outs = [torch.empty((prm["n_frames"], 1, prm["side"], prm["side"]), dtype=torch.float32, device="cuda")
                for prm in params]
        b_units = float(sum(prm["n_atoms"] * prm["n_frames"] * prm["side"] ** 2 for prm in params))
        xs.intensity_batched(trajs, grids, "bf16", outs)     # builds and captures the graph
        ctx.sync_status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            xs.intensity_batched(trajs, grids, "bf16", outs)  # graph replay
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        b_ms = e0.elapsed_time(e1) / 2
        # the autotuner: tile kind x chunk length per shape bucket, then the
        # same call again with every trajectory on its bucket's choice
        t_tune = time.perf_counter()
        xs.tune_batched(trajs, grids, "bf16")
        t_tune = time.perf_counter() - t_tune
        choices = [xs.tuned_choice(prm["n_atoms"], g, "bf16") for prm, g in zip(params, grids)]
        xs.intensity_batched(trajs, grids, "bf16", outs)     # captures the tuned graph
        ctx.sync_status()
        e0.record(stream)
        for _ in range(2):
            xs.intensity_batched(trajs, grids, "bf16", outs)
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        bt_ms = e0.elapsed_time(e1) / 2
        # the whole pipeline: each trajectory's g2 on 64 log-spaced delays and
        # XSVS contrast on 1-2-5 windows over unit rings, in the same graph
        taus_b = [[int(t) for t in wl.log_delays(prm["n_frames"], 64)] for prm in params]
        Ks_b = [[int(k) for k in wl.window_list_125(prm["n_frames"])] for prm in params]
        R_b = [wl.rings_for_plane(g) for g in grids]
        xs.xpcs_batched(trajs, grids, taus_b, Ks_b, R_b, "bf16", outs=outs)   # captures the graph
        ctx.sync_status()
        e0.record(stream)
        for _ in range(2):
            res_b = xs.xpcs_batched(trajs, grids, taus_b, Ks_b, R_b, "bf16", outs=outs)
        e1.record(stream)
        e1.synchronize()
        ctx.sync_status()
        p_ms = e0.elapsed_time(e1) / 2
        line["batched"] = {"workload": "64 ideal-gas trajectories, N log-uniform 2e3-5e5, T 100-2000, "
                                       "planes 64^2-256^2, split BF16, one persistent launch per call",
                           "units": b_units, "ms_per_call": b_ms, "value": b_units / (b_ms * 1e-3), "unit": METRIC,
                           "tiles": "default rule: 128 x 64 tiles where n_y <= 64, else 128 x 128",
                           "tuned": {"ms_per_call": bt_ms, "value": b_units / (bt_ms * 1e-3), "unit": METRIC,
                                     "tuning_s": t_tune,
                                     "tile_kinds": {"128x128": sum(1 for c in choices if c[0] == 0),
                                                    "128x64": sum(1 for c in choices if c[0] == 1)},
                                     "chunks": {str(k): sum(1 for c in choices if c[1] == k) for k in (16, 32, 64)}},
                           "pipeline": {"what": "intensity, then per trajectory g2 (64 log delays) and XSVS "
                                                "(1-2-5 windows, unit rings), one captured graph per call",
                                        "ms_per_call": p_ms, "value": b_units / (p_ms * 1e-3), "unit": METRIC,
                                        "correlation_ms": p_ms - b_ms}}
        del res_b
        del trajs, outs
        torch.cuda.empty_cache()

    # ---- the 4,000-atom workload on the FP32 path and the 3.2-million-atom
    # crystal (512^2 plane streamed from host memory, 128^3 volume, g2 and XSVS
    # at 10,000 frames of 512^2) ------------------------------------------------
    cfg_keep = {}
    if not args.no_configs and rank == 0:
        line["configs"], cfg_keep = config_entries(xs, ctx, stream, _peaks())

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N = 1) ----
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle

        oracle.build()
        m = grid.miller()
        sel = np.arange(0, m.shape[0], 2)
        t0 = time.perf_counter()
        ref = oracle.intensity(traj.pos[:1], traj.f, traj.box, m[sel])
        dt = time.perf_counter() - t0
        got = I_step.view(T, -1)[0].cpu().numpy().astype(np.float64)[sel]
        nz = np.any(m[sel] != 0, axis=1)
        e_I = float(np.linalg.norm(got[nz] - ref[0, nz]) / np.linalg.norm(ref[0, nz]))
        d_I = np.abs(got[nz] - ref[0, nz])
        mean_ref = float(ref[0, nz].mean())
        e_pix = float(np.max(d_I / np.maximum(ref[0, nz], mean_ref)))
        mean_dev = float(d_I.max() / mean_ref)
        line["cpu_baseline"] = {"value": traj.n_atoms * sel.size / dt, "unit": METRIC,
                                "cores": oracle.max_threads(), "kind": "oracle",
                                "sample": f"frame 0, {sel.size} of {m.shape[0]} pixels (every 2nd), "
                                          f"{traj.n_atoms} atoms, {dt:.1f} s"}
        # g2 and the XSVS contrast of the last timed step against the oracle's
        # g2 and contrast of the kernel's own intensity (stage parity)
        g_k, _, beta_k = res
        pix_g = np.arange(0, m.shape[0], 8)
        Ih = I_step.view(T, -1)[:, torch.from_numpy(pix_g).cuda()].cpu().numpy()
        gref, mref = oracle.g2(Ih, taus)
        gk = g_k.cpu().numpy()[:, pix_g]
        nzg = np.any(m[pix_g] != 0, axis=1)
        e_g2 = float(np.linalg.norm(gk[:, nzg] - gref[:, nzg]) / np.linalg.norm(gref[:, nzg]))
        bright = nzg & (mref >= 1e-2 * mref[nzg].mean())
        e_g2_pix = float(np.max(np.abs(gk[:, bright] - gref[:, bright]) / np.abs(gref[:, bright])))
        rings = oracle.ring_index(box, m, 1.0, R)
        bref, cref = oracle.xsvs_contrast(I_step.view(T, -1).cpu().numpy(), Ks, rings, R)
        okr = cref >= 8
        bk = beta_k.cpu().numpy()
        e_beta = float(np.max(np.abs(bk[:, okr] - bref[:, okr]) / np.abs(bref[:, okr])))
        if keep_tables:
            # frame 0 from both table builders against the same oracle sample
            tb = line["next_rows"]["table_builders"]
            for name in ("rec", "exact"):
                gv = keep_tables[name].astype(np.float64)[sel]
                tb[f"e_I_frame0_{name}"] = float(np.linalg.norm(gv[nz] - ref[0, nz]) / np.linalg.norm(ref[0, nz]))
        line["accuracy"] = {
            "e_I_frame0": e_I, "e_pix_frame0": e_pix, "max_abs_dI_over_mean_frame0": mean_dev,
            "e_g2": e_g2, "e_g2_max_rel_bright": e_g2_pix, "g2_pixels": int(nzg.sum()),
            "g2_bright_pixels": int(bright.sum()), "e_beta": e_beta, "beta_entries": int(okr.sum() * len(Ks)),
            "against": "FP64 oracle: intensity on the cpu_baseline sample (frame 0); g2 on every 8th pixel and "
                       "beta on every (K, ring) with >= 8 pixels, from the kernel's own intensity",
            "definitions": "e_I = ||dI||_2/||I_ref||_2 over q != 0; e_pix = max |dI| / max(I_ref, mean I_ref); "
                           "e_g2 = ||dg2||_2/||g2_ref||_2; e_beta = max relative error"}
        # one host core on a smaller sample, and the 4,000-atom workload in full
        sel1 = np.arange(0, m.shape[0], 32)
        t0 = time.perf_counter()
        oracle.intensity(traj.pos[:1], traj.f, traj.box, m[sel1], threads=1)
        dt1 = time.perf_counter() - t0
        line["cpu_baseline"]["single_core"] = {"value": traj.n_atoms * sel1.size / dt1, "unit": METRIC,
                                               "sample": f"frame 0, {sel1.size} pixels (every 32nd)"}
        t0c, g0 = wl.config0()
        t0 = time.perf_counter()
        ref0 = oracle.intensity(t0c.pos, t0c.f, t0c.box, g0.miller())
        dt0 = time.perf_counter() - t0
        if cfg_keep:
            config_accuracy(line["configs"], cfg_keep, ref0)
        line["cpu_baseline"]["config_4000_atoms_full"] = {
            "value": t0c.n_atoms * g0.n_pixels * t0c.pos.shape[0] / dt0, "unit": METRIC, "seconds": dt0,
            "workload": "4,000 atoms, 10 frames, 64^2 plane, all host cores"}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("--steps must be at least 1 and --warmup at least 0")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
