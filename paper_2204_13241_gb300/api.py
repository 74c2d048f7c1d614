"""PyTorch-facing calls of the library: argument marshalling only.

Every computation runs in libxs.so (include/xs_api.h); PyTorch supplies
device memory (through its caching allocator), the current CUDA stream and
autograd plumbing.  Tensors must be contiguous float32 (positions, form
factors, intensities, amplitudes).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as nat
from .workloads import QGrid as GridSpec


def _box(box) -> nat.Box:
    h = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(9))
    b = nat.Box()
    for i in range(9):
        b.h[i] = float(h[i])
    return b


def _grid(grid) -> nat.QGrid:
    if isinstance(grid, GridSpec):
        t = grid.as_tuple()
    else:
        t = tuple(int(v) for v in grid)
    return nat.QGrid(*t)


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, name: str, dtype=torch.float32, cuda: Optional[bool] = True):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if cuda is True and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if cuda is False and t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")


class Context:
    """One libxs context per CUDA device; workspace comes from PyTorch's
    caching allocator."""

    _per_device: dict[int, "Context"] = {}

    def __init__(self, device: Optional[int] = None):
        self.lib = nat.load()
        self.device = torch.cuda.current_device() if device is None else int(device)

        def _alloc(nbytes, _ctx):
            with torch.cuda.device(self.device):
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device)

        def _free(ptr, _ctx):
            with torch.cuda.device(self.device):
                torch.cuda.caching_allocator_delete(int(ptr))

        self._fns = (nat.ALLOC_FN(_alloc), nat.FREE_FN(_free))
        self._alloc = nat.Allocator(self._fns[0], self._fns[1], None)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(self.lib.xs_context_create(ctypes.byref(self._alloc), ctypes.byref(handle)))
        self.handle = handle

    @classmethod
    def get(cls, device: Optional[int] = None) -> "Context":
        dev = torch.cuda.current_device() if device is None else int(device)
        ctx = cls._per_device.get(dev)
        if ctx is None:
            ctx = cls(dev)
            cls._per_device[dev] = ctx
        return ctx

    def close(self):
        if self.handle:
            with torch.cuda.device(self.device):
                self.lib.xs_context_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def sync_status(self) -> None:
        nat.check(self.lib.xs_sync_status(self.handle, _stream()))

    def set_wait_timeout_ns(self, ns: int) -> None:
        nat.check(self.lib.xs_set_wait_timeout_ns(self.handle, int(ns)))

    def set_table_builder(self, exact: bool) -> None:
        """False: tensor-core tables from FP32 seeds and rotations (default);
        True: every entry from FP64 sincospi of its exact turn count."""
        nat.check(self.lib.xs_set_table_builder(self.handle, 1 if exact else 0))

    def profile(self, on: bool) -> None:
        """Bracket every launch group with CUDA events on its stream."""
        nat.check(self.lib.xs_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, prefix: str = "") -> tuple[float, int]:
        """(device milliseconds, kernels) of launch groups named `prefix`* since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        nat.check(self.lib.xs_profile_read(self.handle, prefix.encode(), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        nat.check(self.lib.xs_launch_count(self.handle, ctypes.byref(n)))
        return n.value


def _traj(pos: torch.Tensor, f: torch.Tensor, box) -> tuple[nat.Traj, bool]:
    if pos.dim() == 2:
        pos = pos.unsqueeze(0)
    if pos.dim() != 3 or pos.shape[-1] != 3:
        raise ValueError("positions must be [T][N][3]")
    host = not pos.is_cuda
    _need(pos, "pos", cuda=not host)
    _need(f, "f", cuda=not host)
    if f.numel() != pos.shape[1]:
        raise ValueError("f must have one entry per atom")
    tr = nat.Traj(pos.data_ptr(), 1 if host else 0, f.data_ptr(), pos.shape[1], pos.shape[0], _box(box))
    return tr, host


def intensity(pos: torch.Tensor, f: torch.Tensor, box, grid, precision: str = "fp16",
              want_amp: bool = False, out: Optional[torch.Tensor] = None,
              amp_out: Optional[torch.Tensor] = None):
    """I(q,t) = |sum_j f_j exp(i q.r_j(t))|^2 on `grid` for every frame
    (Sec. 3.1, Algorithm 1).  Returns I [T][nz][ny][nx] (and the amplitude
    [T][nz][ny][nx][2] when want_amp).  Host positions are streamed."""
    tr, host = _traj(pos, f, box)
    g = _grid(grid)
    shape = (int(tr.n_frames), g.nz, g.ny, g.nx)
    dev = torch.device("cuda", torch.cuda.current_device()) if not host else torch.device("cpu")
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=dev, pin_memory=host)
    _need(out, "out", cuda=None)
    if want_amp and amp_out is None:
        amp_out = torch.empty(shape + (2,), dtype=torch.float32, device=dev, pin_memory=host)
    if amp_out is not None:
        _need(amp_out, "amp_out", cuda=None)
    ctx = Context.get()
    nat.check(ctx.lib.xs_intensity(ctx.handle, ctypes.byref(tr), ctypes.byref(g), nat.PRECISIONS[precision],
                                   _ptr(out), _ptr(amp_out), _stream()))
    return (out, amp_out) if want_amp else out


def intensity_species(pos: torch.Tensor, f: torch.Tensor, species, coef, box, grid, precision: str = "fp16",
                      want_amp: bool = False):
    """I(q,t) with q-dependent form factors per species (Sec. 2.1):
    S = sum_j f_j F_{s_j}(q) exp(i q.r_j); `species` int [N] (host), `coef`
    float64 [n_species][9] Gaussian-sum coefficients (a1, b1, .., a4, b4, c)."""
    tr, host = _traj(pos, f, box)
    if host:
        raise ValueError("the species path takes device positions")
    sp = np.ascontiguousarray(np.asarray(species, dtype=np.int32).reshape(-1))
    cf = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, 9))
    if sp.size != tr.n_atoms:
        raise ValueError("one species per atom")
    g = _grid(grid)
    shape = (int(tr.n_frames), g.nz, g.ny, g.nx)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    amp = torch.empty(shape + (2,), dtype=torch.float32, device="cuda") if want_amp else None
    ctx = Context.get()
    nat.check(ctx.lib.xs_intensity_species(ctx.handle, ctypes.byref(tr), sp.ctypes.data_as(ctypes.c_void_p),
                                           cf.shape[0], cf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(g),
                                           nat.PRECISIONS[precision], out.data_ptr(), _ptr(amp), _stream()))
    return (out, amp) if want_amp else out


def intensity_points(pos: torch.Tensor, f: torch.Tensor, box, miller, precision: str = "fp16",
                     want_amp: bool = False):
    """I at arbitrary reciprocal-lattice points `miller` int [P][3] (host),
    for every frame: returns I [T][P] (and the amplitude [T][P][2])."""
    tr, host = _traj(pos, f, box)
    if host:
        raise ValueError("the point path takes device positions")
    m = np.ascontiguousarray(np.asarray(miller, dtype=np.int32).reshape(-1, 3))
    shape = (int(tr.n_frames), m.shape[0])
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    amp = torch.empty(shape + (2,), dtype=torch.float32, device="cuda") if want_amp else None
    ctx = Context.get()
    nat.check(ctx.lib.xs_intensity_points(ctx.handle, ctypes.byref(tr), m.ctypes.data_as(ctypes.c_void_p),
                                          m.shape[0], nat.PRECISIONS[precision], _ptr(out), _ptr(amp), _stream()))
    return (out, amp) if want_amp else out


def intensity_fft(pos: torch.Tensor, f: torch.Tensor, box, grid, n_grid: int, eta: float, k_cut: int = 0,
                  want_amp: bool = False):
    """I by the FFT-based method (Sec. 3.2, Algorithm 2) on an n_grid^3 grid,
    reported on `grid`; a cross-check of the direct method."""
    tr, host = _traj(pos, f, box)
    if host:
        raise ValueError("the FFT path takes device positions")
    g = _grid(grid)
    shape = (int(tr.n_frames), g.nz, g.ny, g.nx)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    amp = torch.empty(shape + (2,), dtype=torch.float32, device="cuda") if want_amp else None
    ctx = Context.get()
    nat.check(ctx.lib.xs_intensity_fft(ctx.handle, ctypes.byref(tr), int(n_grid), float(eta), int(k_cut),
                                       ctypes.byref(g), out.data_ptr(), _ptr(amp), _stream()))
    return (out, amp) if want_amp else out


def ewald_points(box, k_in, nx0: int, nx: int, ny0: int, ny: int):
    """Reciprocal-lattice points of the Ewald-sphere slice over a detector
    window (host helper of the library): (miller int32 [nx*ny][3], valid bool)."""
    b = _box(box)
    k = np.ascontiguousarray(np.asarray(k_in, dtype=np.float64).reshape(3))
    m = np.zeros((nx * ny, 3), dtype=np.int32)
    v = np.zeros(nx * ny, dtype=np.uint8)
    nat.check(nat.load().xs_ewald_points(ctypes.byref(b), k.ctypes.data_as(ctypes.c_void_p), nx0, nx, ny0, ny,
                                         m.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p)))
    return m, v.astype(bool)


def intensity_batched(trajs: Sequence[tuple], grids: Sequence, precision: str = "bf16",
                      outs: Optional[Sequence[torch.Tensor]] = None):
    """Many trajectories (pos, f, box) on their own grids in one call."""
    n = len(trajs)
    arr_t = (nat.Traj * n)()
    arr_g = (nat.QGrid * n)()
    keep = []
    for i, (pos, f, box) in enumerate(trajs):
        tr, host = _traj(pos, f, box)
        if host:
            raise ValueError("batched trajectories need device positions")
        arr_t[i] = tr
        arr_g[i] = _grid(grids[i])
    if outs is None:
        outs = [torch.empty((int(arr_t[i].n_frames), arr_g[i].nz, arr_g[i].ny, arr_g[i].nx), dtype=torch.float32,
                            device="cuda") for i in range(n)]
    ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    keep.append(ptrs)
    ctx = Context.get()
    nat.check(ctx.lib.xs_intensity_batched(ctx.handle, arr_t, arr_g, n, nat.PRECISIONS[precision], ptrs, _stream()))
    return outs


def xpcs_batched(trajs: Sequence[tuple], grids: Sequence, taus: Sequence, Ks: Sequence, n_rings: Sequence[int],
                 precision: str = "bf16", ring_width: float = 1.0, outs: Optional[Sequence[torch.Tensor]] = None):
    """Batched pipeline: intensities of many trajectories (pos, f, box) on their
    own grids, then each one's g2 on taus[i] (Sec. 2.3 Eq. g2_def) and XSVS
    contrast on Ks[i] over n_rings[i] rings (Eqs. inte_Iq, bq_Iq), in one call
    (one captured graph on the split paths).  Returns (I, g2, mean, beta,
    ring counts) lists."""
    n = len(trajs)
    arr_t = (nat.Traj * n)()
    arr_g = (nat.QGrid * n)()
    for i, (pos, f, box) in enumerate(trajs):
        tr, host = _traj(pos, f, box)
        if host:
            raise ValueError("batched trajectories need device positions")
        arr_t[i] = tr
        arr_g[i] = _grid(grids[i])
    if outs is None:
        outs = [torch.empty((int(arr_t[i].n_frames), arr_g[i].nz, arr_g[i].ny, arr_g[i].nx), dtype=torch.float32,
                            device="cuda") for i in range(n)]
    reqs = (nat.CorrRequest * n)()
    keep, g2s, means, betas, counts = [], [], [], [], []
    for i in range(n):
        P = arr_g[i].nx * arr_g[i].ny * arr_g[i].nz
        t = np.ascontiguousarray(taus[i], dtype=np.int32)
        k = np.ascontiguousarray(Ks[i], dtype=np.int32)
        g = torch.empty((t.size, P), dtype=torch.float64, device="cuda")
        m = torch.empty((P,), dtype=torch.float64, device="cuda")
        b = torch.empty((k.size, int(n_rings[i])), dtype=torch.float64, device="cuda")
        c = np.zeros(int(n_rings[i]), dtype=np.int32)
        keep += [t, k]
        reqs[i] = nat.CorrRequest(t.ctypes.data if t.size else None, t.size, g.data_ptr() if t.size else None,
                                  m.data_ptr(), k.ctypes.data if k.size else None, k.size, float(ring_width),
                                  int(n_rings[i]), b.data_ptr() if b.numel() else None,
                                  c.ctypes.data if c.size else None)
        g2s.append(g)
        means.append(m)
        betas.append(b)
        counts.append(c)
    ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    ctx = Context.get()
    nat.check(ctx.lib.xs_xpcs_batched(ctx.handle, arr_t, arr_g, n, nat.PRECISIONS[precision], ptrs, reqs, _stream()))
    return outs, g2s, means, betas, counts


def tune(pos: torch.Tensor, f: torch.Tensor, box, grid, precision: str = "fp16") -> None:
    tr, host = _traj(pos, f, box)
    g = _grid(grid)
    ctx = Context.get()
    nat.check(ctx.lib.xs_tune(ctx.handle, ctypes.byref(tr), ctypes.byref(g), nat.PRECISIONS[precision], _stream()))


def tuned_choice(n_atoms: int, grid, precision: str = "fp16") -> tuple[int, int]:
    """(tile kind, chunk stages) the split path uses for this shape: 0 is the
    128 x 128 tile, 1 the 128 x 64 tile (see xs_tune)."""
    g = _grid(grid)
    k, c = ctypes.c_int32(), ctypes.c_int32()
    ctx = Context.get()
    nat.check(ctx.lib.xs_tuned_choice(ctx.handle, int(n_atoms), ctypes.byref(g), nat.PRECISIONS[precision],
                                      ctypes.byref(k), ctypes.byref(c)))
    return int(k.value), int(c.value)


def tune_batched(trajs: Sequence[tuple], grids: Sequence, precision: str = "bf16") -> None:
    """Runs the tuner once per distinct shape bucket of a batch (atoms by
    powers of two after padding, grid), so that every trajectory of later
    batched calls uses its bucket's tile kind and chunk length."""
    seen = set()
    for (pos, f, box), grid in zip(trajs, grids):
        n = int(pos.shape[1])
        npad = max(64, (n + 63) // 64 * 64)
        key = (npad.bit_length() - 1, tuple(_grid_tuple(grid)))
        if key in seen:
            continue
        seen.add(key)
        tune(pos, f, box, grid, precision)


def _grid_tuple(grid):
    g = _grid(grid)
    return (g.nx0, g.nx, g.ny0, g.ny, g.nz0, g.nz)


def g2(I: torch.Tensor, taus: Sequence[int], want_mean: bool = True):
    """g2(q,tau) per pixel (Sec. 2.3 Eq. g2_def) of I [T][...]; returns
    (g2 float64 [n_tau][P], mean float64 [P])."""
    _need(I, "I")
    T = I.shape[0]
    P = I.numel() // max(T, 1)
    t = np.ascontiguousarray(np.asarray(taus, dtype=np.int32))
    out = torch.empty((t.size, P), dtype=torch.float64, device=I.device)
    mean = torch.empty((P,), dtype=torch.float64, device=I.device) if want_mean else None
    ctx = Context.get()
    nat.check(ctx.lib.xs_g2(ctx.handle, I.data_ptr(), T, P, t.ctypes.data_as(ctypes.c_void_p), t.size,
                            out.data_ptr(), _ptr(mean), _stream()))
    return out, mean


def xsvs_contrast(I: torch.Tensor, grid, box, Ks: Sequence[int], n_rings: int, ring_width: float = 1.0):
    """beta_K(ring) (Sec. 2.3 Eqs. inte_Iq, bq_Iq) of I [T][nz][ny][nx];
    returns (beta float64 [n_K][n_rings], pixels per ring int32 [n_rings])."""
    _need(I, "I")
    g = _grid(grid)
    b = _box(box)
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    beta = torch.empty((k.size, n_rings), dtype=torch.float64, device=I.device)
    counts = np.zeros(n_rings, dtype=np.int32)
    ctx = Context.get()
    nat.check(ctx.lib.xs_xsvs_contrast(ctx.handle, I.data_ptr(), I.shape[0], ctypes.byref(g), ctypes.byref(b),
                                       k.ctypes.data_as(ctypes.c_void_p), k.size, float(ring_width), int(n_rings),
                                       beta.data_ptr(), counts.ctypes.data_as(ctypes.c_void_p), _stream()))
    return beta, counts


def isf(amp: torch.Tensor, taus: Sequence[int], sum_f2: float, want_hat: bool = True):
    """Intermediate scattering function (Sec. 2.3 Eqs. Fq_pq, norm_Fq) of the
    amplitudes amp [T][...][2] written by `intensity(..., want_amp=True)`;
    returns (F, F_hat) as complex128 [n_tau][P] (F_hat None unless want_hat)."""
    _need(amp, "amp")
    if amp.shape[-1] != 2:
        raise ValueError("amp must end in a (re, im) axis of 2")
    T = amp.shape[0]
    P = amp.numel() // max(2 * T, 1)
    t = np.ascontiguousarray(np.asarray(taus, dtype=np.int32))
    F = torch.empty((t.size, P, 2), dtype=torch.float64, device=amp.device)
    Fh = torch.empty((t.size, P, 2), dtype=torch.float64, device=amp.device) if want_hat else None
    ctx = Context.get()
    nat.check(ctx.lib.xs_isf(ctx.handle, amp.data_ptr(), T, P, t.ctypes.data_as(ctypes.c_void_p), t.size,
                             float(sum_f2), F.data_ptr(), _ptr(Fh), _stream()))
    F = torch.view_as_complex(F)
    return F, (torch.view_as_complex(Fh) if want_hat else None)


def contrast_from_isf(Fhat: torch.Tensor, grid, box, Ks: Sequence[int], n_rings: int, ring_width: float = 1.0):
    """beta_K / beta_0 per ring predicted from F_hat (Sec. 2.3 Eq. beta_alt_int,
    K-frame form); Fhat complex128 [Kmax][P] on the delays 0..Kmax-1.
    Returns (ratio float64 [n_K][n_rings], pixels per ring int32 [n_rings])."""
    if Fhat.dtype != torch.complex128 or not Fhat.is_cuda or not Fhat.is_contiguous():
        raise ValueError("Fhat must be a contiguous complex128 CUDA tensor")
    g = _grid(grid)
    b = _box(box)
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    out = torch.empty((k.size, n_rings), dtype=torch.float64, device=Fhat.device)
    counts = np.zeros(n_rings, dtype=np.int32)
    ctx = Context.get()
    nat.check(ctx.lib.xs_contrast_from_isf(ctx.handle, Fhat.data_ptr(), Fhat.shape[0], ctypes.byref(g),
                                           ctypes.byref(b), k.ctypes.data_as(ctypes.c_void_p), k.size,
                                           float(ring_width), int(n_rings), out.data_ptr(),
                                           counts.ctypes.data_as(ctypes.c_void_p), _stream()))
    return out, counts


def xsvs_partial(I: torch.Tensor, ring, n_rings: int, Ks: Sequence[int]):
    """Per-(K, window, ring) sums (sum I_K, sum I_K^2) over the pixels of a
    shard, I [T][P_shard], ring int [P_shard] (host); returns (sums float64
    [n_kw][n_rings][2] on the device, counts int64 [n_rings] on the host)."""
    _need(I, "I")
    T = I.shape[0]
    P = I.numel() // max(T, 1)
    rg = np.ascontiguousarray(np.asarray(ring, dtype=np.int32).reshape(-1))
    if rg.size != P:
        raise ValueError("one ring label per pixel")
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    n_kw = int(sum(T // int(K) for K in k))
    sums = torch.zeros((n_kw, n_rings, 2), dtype=torch.float64, device=I.device)
    counts = np.zeros(n_rings, dtype=np.int64)
    ctx = Context.get()
    nat.check(ctx.lib.xs_xsvs_partial(ctx.handle, I.data_ptr(), T, P, rg.ctypes.data_as(ctypes.c_void_p), int(n_rings),
                                      k.ctypes.data_as(ctypes.c_void_p), k.size, sums.data_ptr() if sums.numel() else None,
                                      counts.ctypes.data_as(ctypes.c_void_p), _stream()))
    return sums, counts


def xsvs_finalize(sums, counts, T: int, Ks: Sequence[int]) -> np.ndarray:
    """beta_K(r) from summed shard sums (host or device array [n_kw][n_rings][2])
    and counts [n_rings] (host, library routine without GPU work)."""
    sm = np.ascontiguousarray(np.asarray(sums.cpu() if hasattr(sums, "cpu") else sums, dtype=np.float64))
    ct = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    n_rings = ct.size
    out = np.zeros((k.size, n_rings), dtype=np.float64)
    nat.check(nat.load().xs_xsvs_finalize(sm.ctypes.data_as(ctypes.c_void_p), ct.ctypes.data_as(ctypes.c_void_p),
                                          int(T), k.ctypes.data_as(ctypes.c_void_p), k.size, n_rings,
                                          out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ring_index(grid, box, ring_width: float, n_rings: int) -> np.ndarray:
    """Ring of every pixel as used by xsvs_contrast (host computation)."""
    g = _grid(grid)
    out = np.zeros(g.nx * g.ny * g.nz, dtype=np.int32)
    lib = nat.load()
    nat.check(lib.xs_ring_index(ctypes.byref(g), ctypes.byref(_box(box)), float(ring_width), int(n_rings),
                                out.ctypes.data_as(ctypes.c_void_p)))
    return out


def intensity_backward(pos: torch.Tensor, f: torch.Tensor, box, grid, amp: torch.Tensor,
                       dL_dI: torch.Tensor) -> torch.Tensor:
    """dL/dr [N][3] for one frame from S (amp [P][2]) and dL/dI [P]."""
    tr, host = _traj(pos, f, box)
    if host:
        raise ValueError("the adjoint needs device positions")
    _need(amp, "amp")
    _need(dL_dI, "dL_dI")
    g = _grid(grid)
    grad = torch.empty((int(tr.n_atoms), 3), dtype=torch.float32, device=pos.device)
    ctx = Context.get()
    nat.check(ctx.lib.xs_intensity_backward(ctx.handle, ctypes.byref(tr), ctypes.byref(g), amp.data_ptr(),
                                            dL_dI.data_ptr(), grad.data_ptr(), _stream()))
    return grad


class IntensityFn(torch.autograd.Function):
    """I(q) of one frame as a differentiable function of positions [N][3].

    forward runs xs_intensity (by default the factorised FP32 path, which
    meets the FP32 accuracy of the plain direct kernel about ten times
    faster) and keeps S; backward runs xs_intensity_backward."""

    @staticmethod
    def forward(ctx, pos, f, box, grid, precision="fp32f"):
        p = pos.detach().contiguous()
        I, amp = intensity(p, f, box, grid, precision, want_amp=True)
        ctx.save_for_backward(p, f, amp)
        ctx.box = box
        ctx.grid = grid
        return I.reshape(-1)

    @staticmethod
    def backward(ctx, grad_I):
        p, f, amp = ctx.saved_tensors
        g = intensity_backward(p, f, ctx.box, ctx.grid, amp.reshape(-1, 2).contiguous(),
                               grad_I.contiguous().to(torch.float32))
        return g.reshape(p.shape), None, None, None, None
